// Shifted solves and moment accumulation (Alg. 1 / Alg. 2 steps 1-2).
//
// All N/2 systems (s_j I - H) Y_j = X, H = A^T A, share one Krylov space per
// right-hand-side column. Since H is real symmetric and X real, the COCG
// iterate of every shifted system is the Lanczos-Galerkin solution
//   Y_j = Q_K (s_j I - T_K)^{-1} e_1 beta_1,
// with Q_K, T_K from real Lanczos on H. The moments only need
//   S_k = 2 Re sum_j w_j m_j^k Y_j = Q_K c_k,  c_k = 2 Re sum_j w_j m_j^k (s_j I - T_K)^{-1} e_1 beta_1,
// so no per-shift n-vector is ever stored:
//   pass 1  Lanczos on H; per (shift, column) the LDL^T pivots of s_j I - T_k
//           give the residual ||r_j|| = beta_{k+1} |e_k^T (s_j I - T_k)^{-1} e_1| beta_1
//           without forming Y_j; stop when all are <= tol_solve * beta_1,
//   tri     per (shift, column) solve (s_j I - T_K) y = beta_1 e_1 by LDL^T
//           (no pivoting: Im s_j != 0 keeps every leading block nonsingular),
//   pass 2  regenerate the same Lanczos vectors (bitwise: same kernels, same
//           explicitly rounded operations), keep them in a panel of P vectors and,
//           once per panel, add S_k += sum_{i in panel} c_{k,i} q_i (the block S is
//           read and written once per P steps, not once per step).
// The SpMM is real (L columns), not complex (2L). Iterations run as CUDA graphs;
// convergence is polled every check_every iterations.
//
// Two vector formats share these kernels (Vec policies below):
//   F64  the Lanczos vectors and the SpMM in FP64 (FP64 precision);
//   DF   double-float: every vector element is an unevaluated sum hi + lo of two FP32
//        numbers, and the SpMM, the vector updates, the dot products and the panel
//        accumulation run on the FP32 pipe with error-free transformations (two_prod,
//        two_sum). The unit roundoff is about 2^-48 instead of 2^-53, and on GB300 the
//        FP32 pipe issues 64 times the FMAs of the FP64 pipe. The scalars of the
//        recurrence (alpha, beta, the LDL^T pivots, the tridiagonal solves, the moment
//        coefficients) and S itself stay FP64. This is the mixed-precision mode; its
//        shifted solves are then checked and, if needed, refined in FP64
//        (refined_filter, at the end of this file).
#include "internal.cuh"

namespace cmsvd {

// ----------------------------------------------------------------------------- complex helpers
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// Smith's division (robust against overflow of |b|^2)
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    } else {
        double r = b.x / b.y, den = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
    }
}
__device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }


// explicitly rounded operations of the vector recurrences: pass 2 repeats pass 1's
// operations exactly, so the regenerated vectors are bitwise equal
// ----------------------------------------------------------------------------- quadrature (Sec. 4)
__global__ void k_quadrature(QuadParams q, double2* quad) {
    const int J = q.N / 2;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const double pi = 3.14159265358979323846;
    const double theta = 2.0 * pi / q.N * (j + 0.5);   // theta_j = 2 pi (j - 1/2) / N, j 1-based
    double gamma, rho;
    if (q.variant == CMSVD_LINEAR) {
        gamma = 0.5 * (q.a * q.a + q.b * q.b);
        rho = 0.5 * (q.b * q.b - q.a * q.a);
    } else {
        gamma = log(q.a) + log(q.b);
        rho = log(q.b) - log(q.a);
    }
    const double c = cos(theta), s = sin(theta);
    const double2 node = make_double2(gamma + rho * c, rho * q.alpha * s);
    const double2 w0 = make_double2(rho / q.N * q.alpha * c, rho / q.N * s);
    double2 shift, weight;
    if (q.variant == CMSVD_LINEAR) {
        shift = node;
        weight = w0;
    } else {
        const double er = exp(node.x);
        shift = make_double2(er * cos(node.y), er * sin(node.y));   // g(t_j) = exp(t_j)
        weight = cmul(w0, shift);                                    // psi_j = omega_j exp(t_j)
    }
    quad[3 * j + 0] = shift;
    quad[3 * j + 1] = weight;
    quad[3 * j + 2] = make_double2(c, q.alpha * s);                  // (node_j - gamma) / rho
}

int quadrature_device(const QuadParams& q, double2* quad, cudaStream_t s) {
    ProfScope ps(CMSVD_PROF_OTHER, s, 48.0 * (q.N / 2), 0.0);
    k_quadrature<<<1, 64, 0, s>>>(q, quad);
    CM_LAUNCH();
    return CMSVD_OK;
}


// ----------------------------------------------------------------------------- vector formats
// One Lanczos vector block is n x L elements of 8 bytes. F64: element (i, l) at i L + l.
// DF: row i holds the L high parts, then the L low parts (FP32), as the double-float SpMM
// reads and writes them.
struct VecF64 {
    using E = double;       // one element
    using Sc = double;      // a scalar multiplier
    static constexpr int kind = SPMM_KIND_F64;
    __device__ __forceinline__ static E ld(const void* p, int64_t i, int l, int L) {
        return static_cast<const double*>(p)[i * L + l];
    }
    __device__ __forceinline__ static void st(void* p, int64_t i, int l, int L, E v) { static_cast<double*>(p)[i * L + l] = v; }
    __device__ __forceinline__ static Sc sc(double b) { return b; }
    __device__ __forceinline__ static E zero() { return 0.0; }
    __device__ __forceinline__ static E from_d(double v) { return v; }
    __device__ __forceinline__ static E axmy(E w, Sc b, E q) { return __fma_rn(-b, q, w); }   // w - b q
    __device__ __forceinline__ static E mul(E w, Sc r) { return __dmul_rn(w, r); }
    struct Dot {                                                                                 // sum x y
        double a = 0.0;
        __device__ __forceinline__ void add(E x, E y) { a = __fma_rn(x, y, a); }
        __device__ __forceinline__ double value() const { return a; }
    };
    struct Acc {                                                                                 // sum c q, c FP64
        double a = 0.0;
        __device__ __forceinline__ void add(double c, E q) { a = __fma_rn(c, q, a); }
        __device__ __forceinline__ double value() const { return a; }
    };
    using Coef = double;
    __device__ __forceinline__ static Coef coef(double c) { return c; }
};

struct VecDF {
    using E = float2;
    using Sc = float2;
    static constexpr int kind = SPMM_KIND_DF;
    __device__ __forceinline__ static E ld(const void* p, int64_t i, int l, int L) {
        const float* f = static_cast<const float*>(p) + i * 2 * L + l;
        return make_float2(f[0], f[L]);
    }
    __device__ __forceinline__ static void st(void* p, int64_t i, int l, int L, E v) {
        float* f = static_cast<float*>(p) + i * 2 * L + l;
        f[0] = v.x;
        f[L] = v.y;
    }
    __device__ __forceinline__ static Sc sc(double b) {
        const float h = __double2float_rn(b);
        return make_float2(h, __double2float_rn(b - (double)h));
    }
    __device__ __forceinline__ static E zero() { return make_float2(0.f, 0.f); }
    __device__ __forceinline__ static E from_d(double v) { return sc(v); }
    // w - b q: b q = p + e with p, e from two_prod and the cross terms; the sum is renormalized
    // with two_sum (cancellation can leave the low part larger than the high part)
    __device__ __forceinline__ static E axmy(E w, Sc b, E q) {
        float p, e;
        two_prod(b.x, q.x, p, e);
        e = __fmaf_rn(b.x, q.y, __fmaf_rn(b.y, q.x, e));
        float s, t;
        two_sum(w.x, -p, s, t);
        t = __fadd_rn(t, __fsub_rn(w.y, e));
        float h, lo;
        two_sum(s, t, h, lo);
        return make_float2(h, lo);
    }
    __device__ __forceinline__ static E mul(E w, Sc r) {
        float p, e;
        two_prod(w.x, r.x, p, e);
        e = __fmaf_rn(w.x, r.y, __fmaf_rn(w.y, r.x, e));
        float h, lo;
        fast_two_sum(p, e, h, lo);   // |e| <= 2^-22 |p|
        return make_float2(h, lo);
    }
    // double-float accumulation of products, flushed into an FP64 sum every 32 terms
    struct Dot {
        float hi = 0.f, lo = 0.f;
        double d = 0.0;
        int cnt = 0;
        __device__ __forceinline__ void add(E x, E y) {
            float p, e, s, t;
            two_prod(x.x, y.x, p, e);
            e = __fmaf_rn(x.x, y.y, __fmaf_rn(x.y, y.x, e));
            two_sum(hi, p, s, t);
            hi = s;
            lo = __fadd_rn(lo, __fadd_rn(t, e));
            if (++cnt == 32) { d += (double)hi + (double)lo; hi = lo = 0.f; cnt = 0; }
        }
        __device__ __forceinline__ double value() const { return d + ((double)hi + (double)lo); }
    };
    using Coef = float2;
    __device__ __forceinline__ static Coef coef(double c) { return sc(c); }
    struct Acc {                     // sum c q over one panel (at most 24 terms)
        float hi = 0.f, lo = 0.f;
        __device__ __forceinline__ void add(Coef c, E q) {
            float p, e, s, t;
            two_prod(c.x, q.x, p, e);
            e = __fmaf_rn(c.x, q.y, __fmaf_rn(c.y, q.x, e));
            two_sum(hi, p, s, t);
            hi = s;
            lo = __fadd_rn(lo, __fadd_rn(t, e));
        }
        __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    };
};

// ----------------------------------------------------------------------------- Lanczos state
enum { C_IT = 0, C_NACT = 1, C_STATUS = 2, C_TICKET = 3, C_IT2 = 4, C_KMAX = 5, C_TICKET2 = 6, C_PANEL = 7,
       C_TICKET3 = 8, C_WORDS = 16 };
enum { ST_BREAKDOWN = 1, ST_NOTCONV = 2 };
// rows a thread loads before it computes in the streaming vector kernels (memory-level parallelism)
constexpr int LZ_ROWS = 4;

struct Lz {
    int64_t n = 0;
    int L = 0, J = 0, Mk = 0, max_iter = 0;
    double tol = 0.0;          // < 0: never converge (norm estimation)
    void* Q[3] = {nullptr, nullptr, nullptr};   // n x L vectors (8 bytes per element, F64 or DF)
    void* U = nullptr;         // m x L
    double* alpha = nullptr;   // [max_iter][L]
    double* beta = nullptr;    // [max_iter+1][L]; beta[0] = ||x||
    double2* dcur = nullptr;   // [J][L]
    double2* tcur = nullptr;   // [J][L]
    double2* Dbuf = nullptr;   // [max_iter][J][L]
    double2* Ybuf = nullptr;   // [max_iter][J][L]
    double* C = nullptr;       // [max_iter][Mk][L]
    int* Kcol = nullptr;       // [L]
    int* active = nullptr;     // [L]
    int* ctrl = nullptr;       // [C_WORDS]
    double* partials = nullptr;// [nblk][L]
    int nblk = 0;
    const double2* quad = nullptr;
    int fault_at = 0;          // > 0: step at which column 0 is flagged as broken down (test hook)
    // pass 2 keeps the vectors q_i of the current panel (P slots of n x L) and folds them
    // into its outputs once per panel. Outputs: 0 = moments into S (Mk coefficients per
    // step and column); 1 = Yacc[r][j][l] += y_{i,j,l} q_i (explicit solutions of all
    // shifts); 2 = correction for shift jsel: columns l and Lorig + l carry Re and Im of
    // the right-hand side, Yacc[r][jsel][l] += y_l q_l + i y_{Lorig+l} q_{Lorig+l}.
    void* panel = nullptr;
    int P = 0;
    int mode = 0;
    double2* Yacc = nullptr;   // [n][Jtot][Lorig]
    int Jtot = 0, Lorig = 0, jsel = 0;
};

static dim3 lz_block(int L) {
    int by = 256 / L;
    if (by < 1) by = 1;
    return dim3(L, by);
}

// Column sums of a (rows x L) quantity: per-block partials, the last block adds
// them in block order (deterministic). Returns true in the last block, where
// sums[tx] (shared) holds the column totals for tx < L.
__device__ bool column_reduce(double v, double* sh, double* partials, int* ticket, int L) {
    const int tx = threadIdx.x, ty = threadIdx.y, by = blockDim.y;
    sh[ty * L + tx] = v;
    __syncthreads();
    if (ty == 0) {
        double acc = 0.0;
        for (int r = 0; r < by; ++r) acc += sh[r * L + tx];
        partials[(size_t)blockIdx.x * L + tx] = acc;
    }
    __threadfence();
    __syncthreads();
    __shared__ int last;
    if (tx == 0 && ty == 0) last = (atomicAdd(ticket, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    if (ty == 0) {
        double acc = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) acc += __ldcg(partials + (size_t)b * L + tx);
        sh[tx] = acc;
    }
    __syncthreads();
    if (tx == 0 && ty == 0) *ticket = 0;
    return true;
}

// start: beta_1 = ||x_l||, q_1 = x / beta_1; resets the pass-1 control words.
__global__ void k_lz_norm0(Lz z, const double* __restrict__ X, int64_t ldx) {
    extern __shared__ double sh[];
    const int l = threadIdx.x;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < z.n; i += (int64_t)gridDim.x * blockDim.y) {
        double x = X[i * ldx + l];
        acc = __fma_rn(x, x, acc);
    }
    if (column_reduce(acc, sh, z.partials, z.ctrl + C_TICKET, z.L)) {
        if (threadIdx.y == 0) {
            double b = sqrt(sh[l]);
            z.beta[l] = b;
            z.active[l] = b > 0.0 ? 1 : 0;
            z.Kcol[l] = 0;
        }
        __syncthreads();
        if (l == 0 && threadIdx.y == 0) {
            int na = 0;
            for (int c = 0; c < z.L; ++c) na += z.active[c];
            z.ctrl[C_IT] = 0;
            z.ctrl[C_NACT] = na;
            z.ctrl[C_STATUS] = 0;
            z.ctrl[C_IT2] = 0;
            z.ctrl[C_KMAX] = 0;
        }
    }
}


template <class V>
__global__ void k_lz_scale0(Lz z, const double* __restrict__ X, int64_t ldx, void* __restrict__ Q0) {
    const int l = threadIdx.x;
    const double b = z.beta[l];
    const bool act = b > 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < z.n; i += (int64_t)gridDim.x * blockDim.y)
        V::st(Q0, i, l, z.L, act ? V::from_d(__ddiv_rn(X[i * ldx + l], b)) : V::zero());
}

// pass 1, part 1: w <- H q_k - beta_k q_{k-1};  alpha_k = q_k^T w
template <class V>
__global__ void k_lz_dot(Lz z, const void* __restrict__ Qk, const void* __restrict__ Qp, void* __restrict__ W) {
    extern __shared__ double sh[];
    if (z.ctrl[C_NACT] == 0) return;
    const int k = z.ctrl[C_IT];
    const int l = threadIdx.x;
    const bool act = z.active[l] != 0;
    const typename V::Sc b = V::sc(k > 0 ? z.beta[(size_t)k * z.L + l] : 0.0);
    typename V::Dot acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.y;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i0 < z.n; i0 += LZ_ROWS * stride) {
        typename V::E w[LZ_ROWS], qp[LZ_ROWS], qk[LZ_ROWS];   // loads of LZ_ROWS rows first
#pragma unroll
        for (int u = 0; u < LZ_ROWS; ++u) {
            const int64_t i = i0 + u * stride;
            w[u] = qp[u] = qk[u] = V::zero();
            if (act && i < z.n) {
                w[u] = V::ld(W, i, l, z.L);
                if (k > 0) qp[u] = V::ld(Qp, i, l, z.L);
                qk[u] = V::ld(Qk, i, l, z.L);
            }
        }
#pragma unroll
        for (int u = 0; u < LZ_ROWS; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= z.n) break;
            typename V::E x = V::zero();
            if (act) {
                x = k > 0 ? V::axmy(w[u], b, qp[u]) : w[u];
                acc.add(qk[u], x);
            }
            V::st(W, i, l, z.L, x);
        }
    }
    if (column_reduce(acc.value(), sh, z.partials, z.ctrl + C_TICKET, z.L)) {
        if (threadIdx.y == 0) z.alpha[(size_t)k * z.L + l] = act ? sh[l] : 0.0;
    }
}

// pass 1, part 2: w <- w - alpha_k q_k;  beta_{k+1} = ||w||; per (shift, column)
// LDL^T pivot d and t = e_k^T (s I - T_k)^{-1} e_1 beta_1; convergence and freezing.
template <class V>
__global__ void k_lz_update(Lz z, const void* __restrict__ Qk, void* __restrict__ W) {
    extern __shared__ double sh[];
    if (z.ctrl[C_NACT] == 0) return;
    const int k = z.ctrl[C_IT];
    const int l = threadIdx.x;
    const bool act = z.active[l] != 0;
    const double a = z.alpha[(size_t)k * z.L + l];
    const typename V::Sc at = V::sc(a);
    typename V::Dot acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.y;
    if (act) {
        for (int64_t i0 = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i0 < z.n; i0 += LZ_ROWS * stride) {
            typename V::E w[LZ_ROWS], qk[LZ_ROWS];
#pragma unroll
            for (int u = 0; u < LZ_ROWS; ++u) {
                const int64_t i = i0 + u * stride;
                w[u] = qk[u] = V::zero();
                if (i < z.n) { w[u] = V::ld(W, i, l, z.L); qk[u] = V::ld(Qk, i, l, z.L); }
            }
#pragma unroll
            for (int u = 0; u < LZ_ROWS; ++u) {
                const int64_t i = i0 + u * stride;
                if (i >= z.n) break;
                const typename V::E x = V::axmy(w[u], at, qk[u]);
                V::st(W, i, l, z.L, x);
                acc.add(x, x);
            }
        }
    }
    if (!column_reduce(acc.value(), sh, z.partials, z.ctrl + C_TICKET, z.L)) return;
    if (threadIdx.y == 0) {
        const double bnext = sqrt(sh[l]);
        if (!act) {
            z.beta[(size_t)(k + 1) * z.L + l] = 0.0;
        } else {
            z.beta[(size_t)(k + 1) * z.L + l] = bnext;
            const double b1 = z.beta[l];
            const double bk = z.beta[(size_t)k * z.L + l];
            bool allconv = z.J > 0 && z.tol >= 0.0;
            bool bad = !isfinite(bnext) || !isfinite(a) || (z.fault_at > 0 && l == 0 && k + 1 == z.fault_at);
            for (int j = 0; j < z.J; ++j) {
                const double2 s = z.quad[3 * j];
                const size_t o = (size_t)j * z.L + l;
                double2 d, t;
                if (k == 0) {
                    d = make_double2(s.x - a, s.y);
                    t = cdiv(make_double2(b1, 0.0), d);
                } else {
                    d = csub(make_double2(s.x - a, s.y), cdiv(make_double2(bk * bk, 0.0), z.dcur[o]));
                    t = cdiv(cscale(z.tcur[o], bk), d);
                }
                z.dcur[o] = d;
                z.tcur[o] = t;
                const double res = bnext * cabs_(t) / b1;
                if (!(res <= z.tol)) allconv = false;
                if (!isfinite(res)) bad = true;
            }
            const bool last_iter = k + 1 >= z.max_iter;
            if (bad) atomicOr(z.ctrl + C_STATUS, ST_BREAKDOWN);
            if (allconv || bad || !(bnext > 0.0) || last_iter) {
                z.active[l] = 0;
                z.Kcol[l] = bad ? k : k + 1;
                if (last_iter && !allconv && z.tol >= 0.0) atomicOr(z.ctrl + C_STATUS, ST_NOTCONV);
            }
        }
    }
    __syncthreads();
    if (l == 0 && threadIdx.y == 0) {
        int na = 0, km = 0;
        for (int c = 0; c < z.L; ++c) {
            na += z.active[c];
            km = max(km, z.Kcol[c]);
        }
        z.ctrl[C_NACT] = na;
        z.ctrl[C_KMAX] = km;
        z.ctrl[C_IT] = k + 1;
    }
}

// pass 1, part 3: q_{k+1} = w / beta_{k+1} (zero for frozen columns)

// pass 1, part 3: q_{k+1} = w (1 / beta_{k+1}) (zero for frozen columns)
template <class V>
__global__ void k_lz_scale(Lz z, void* __restrict__ W) {
    const int kk = z.ctrl[C_IT];   // already k+1
    const int l = threadIdx.x;
    const bool act = z.active[l] != 0;
    const typename V::Sc r = V::sc(act ? __drcp_rn(z.beta[(size_t)kk * z.L + l]) : 0.0);
    const int64_t stride = (int64_t)gridDim.x * blockDim.y;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i0 < z.n; i0 += LZ_ROWS * stride) {
        typename V::E w[LZ_ROWS];
#pragma unroll
        for (int u = 0; u < LZ_ROWS; ++u) {
            const int64_t i = i0 + u * stride;
            w[u] = (act && i < z.n) ? V::ld(W, i, l, z.L) : V::zero();
        }
#pragma unroll
        for (int u = 0; u < LZ_ROWS; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < z.n) V::st(W, i, l, z.L, act ? V::mul(w[u], r) : V::zero());
        }
    }
}

// tridiagonal solves: one thread per (shift j, column l); y_i stored in Ybuf
__global__ void k_tri_solve(Lz z) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= z.J * z.L) return;
    const int j = idx / z.L, l = idx % z.L;
    const int K = z.Kcol[l];
    if (K <= 0) return;
    const double2 s = z.quad[3 * j];
    const size_t JL = (size_t)z.J * z.L, o = (size_t)j * z.L + l;
    const double b1 = z.beta[l];
    double2 d = make_double2(0, 0), t = make_double2(0, 0);
    for (int i = 0; i < K; ++i) {
        const double a = z.alpha[(size_t)i * z.L + l];
        if (i == 0) {
            d = make_double2(s.x - a, s.y);
            t = cdiv(make_double2(b1, 0.0), d);
        } else {
            const double bi = z.beta[(size_t)i * z.L + l];
            d = csub(make_double2(s.x - a, s.y), cdiv(make_double2(bi * bi, 0.0), d));
            t = cdiv(cscale(t, bi), d);
        }
        z.Dbuf[i * JL + o] = d;
        z.Ybuf[i * JL + o] = t;
    }
    // back substitution: y_K = t_K, y_i = t_i + (beta_{i+1} / d_i) y_{i+1}
    double2 y = z.Ybuf[(size_t)(K - 1) * JL + o];
    for (int i = K - 2; i >= 0; --i) {
        const double bn = z.beta[(size_t)(i + 1) * z.L + l];
        y = cadd(z.Ybuf[i * JL + o], cmul(cdiv(make_double2(bn, 0.0), z.Dbuf[i * JL + o]), y));
        z.Ybuf[i * JL + o] = y;
    }
}

// c_{m,i,l} = 2 Re sum_j w_j m_j^m y_{i,j,l}; zero beyond the column's K
__global__ void k_tri_coef(Lz z, int Kmax) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Kmax * z.L) return;
    const int i = (int)(idx / z.L), l = (int)(idx % z.L);
    const size_t JL = (size_t)z.J * z.L;
    double* c = z.C + (size_t)i * z.Mk * z.L + l;
    for (int m = 0; m < z.Mk; ++m) c[(size_t)m * z.L] = 0.0;
    if (i >= z.Kcol[l]) return;
    for (int j = 0; j < z.J; ++j) {
        double2 f = z.quad[3 * j + 1];
        const double2 sc = z.quad[3 * j + 2];
        const double2 y = z.Ybuf[i * JL + (size_t)j * z.L + l];
        for (int m = 0; m < z.Mk; ++m) {
            c[(size_t)m * z.L] += 2.0 * (f.x * y.x - f.y * y.y);
            f = cmul(f, sc);
        }
    }
}


// pass 2, one step: copy q_i into panel slot i mod P, then q_{i+1} from the stored alpha, beta
// with the same rounded operations as pass 1.
template <class V>
__global__ void k_lz2_step(Lz z, const void* __restrict__ Qk, const void* __restrict__ Qp, void* __restrict__ W) {
    const int i = z.ctrl[C_IT2];
    if (i >= z.ctrl[C_KMAX]) return;
    const int l = threadIdx.x;
    const int K = z.Kcol[l];
    const bool live = i < K;
    const bool next = i + 1 < K;
    const typename V::Sc at = V::sc(z.alpha[(size_t)i * z.L + l]);
    const typename V::Sc bt = V::sc(i > 0 ? z.beta[(size_t)i * z.L + l] : 0.0);
    const typename V::Sc rt = V::sc(next ? __drcp_rn(z.beta[(size_t)(i + 1) * z.L + l]) : 0.0);
    void* slot = static_cast<char*>(z.panel) + (size_t)(i % z.P) * z.n * z.L * 8;
    const int64_t stride = (int64_t)gridDim.x * blockDim.y;
    for (int64_t r0 = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r0 < z.n; r0 += LZ_ROWS * stride) {
        typename V::E q[LZ_ROWS], w[LZ_ROWS], qp[LZ_ROWS];
#pragma unroll
        for (int u = 0; u < LZ_ROWS; ++u) {
            const int64_t r = r0 + u * stride;
            q[u] = w[u] = qp[u] = V::zero();
            if (r < z.n) {
                q[u] = V::ld(Qk, r, l, z.L);
                if (next) {
                    w[u] = V::ld(W, r, l, z.L);
                    if (i > 0) qp[u] = V::ld(Qp, r, l, z.L);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < LZ_ROWS; ++u) {
            const int64_t r = r0 + u * stride;
            if (r >= z.n) break;
            V::st(slot, r, l, z.L, live ? q[u] : V::zero());
            typename V::E x = V::zero();
            if (next) {
                x = w[u];
                if (i > 0) x = V::axmy(x, bt, qp[u]);
                x = V::axmy(x, at, q[u]);
                x = V::mul(x, rt);
            }
            V::st(W, r, l, z.L, x);
        }
    }
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) last = (atomicAdd(z.ctrl + C_TICKET2, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (last && threadIdx.x == 0 && threadIdx.y == 0) {
        z.ctrl[C_TICKET2] = 0;
        z.ctrl[C_IT2] = i + 1;
    }
}

// Panel fold: the steps [C_PANEL, C_IT2) sit in slots 0..cnt-1 (a panel starts at a
// multiple of P). Per output column l there are kc coefficient rows c (below); groups of
// PANEL_G rows are staged in shared memory and folded into register accumulators (one per
// row c) over the cnt vectors, then added to the FP64 outputs. The last block advances
// C_PANEL.
//   mode 0: c = m < Mk,        S[r][m L + l] += sum_t c_{t,m,l} q_t[r, l]
//   mode 1: c = 2 j + {re, im}, Yacc[r][j][l] += sum_t y_{t,j,l} q_t[r, l]
//   mode 2: c = (y1.re, y1.im, y2.re, y2.im) of the columns l and Lorig + l,
//           Yacc[r][jsel][l] += sum_t y1 q_t[r, l] + i y2 q_t[r, Lorig + l]
constexpr int PANEL_G = 16;
template <class V, int MODE>
__global__ void k_panel(Lz z, double* __restrict__ S, int64_t lds) {
    using Coef = typename V::Coef;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Coef* cs = reinterpret_cast<Coef*>(smem_raw);       // [t][c - c0][l]
    const int i0 = z.ctrl[C_PANEL], i1 = z.ctrl[C_IT2];
    const int cnt = i1 - i0;
    const int L = z.L;
    const int Lo = MODE == 2 ? z.Lorig : L;
    const int kc = MODE == 0 ? z.Mk : (MODE == 1 ? 2 * z.J : 4);
    const size_t JL = (size_t)z.J * L;
    const int nthr = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int l = threadIdx.x;
    const size_t slot_stride = (size_t)z.n * L * 8;
    for (int c0 = 0; c0 < kc && cnt > 0; c0 += PANEL_G) {
        const int g = kc - c0 < PANEL_G ? kc - c0 : PANEL_G;
        __syncthreads();
        for (int e = tid; e < cnt * g * Lo; e += nthr) {
            const int t = e / (g * Lo), c = c0 + (e / Lo) % g, ll = e % Lo;
            const int step = i0 + t;
            double v = 0.0;
            if (MODE == 0) {
                v = z.C[((size_t)step * z.Mk + c) * L + ll];
            } else if (MODE == 1) {
                if (step < z.Kcol[ll]) {
                    const double2 y = z.Ybuf[step * JL + (size_t)(c >> 1) * L + ll];
                    v = (c & 1) ? y.y : y.x;
                }
            } else {
                const int col = c < 2 ? ll : z.Lorig + ll;
                if (step < z.Kcol[col]) {
                    const double2 y = z.Ybuf[step * JL + col];
                    v = (c & 1) ? y.y : y.x;
                }
            }
            cs[((size_t)t * g + (c - c0)) * Lo + ll] = V::coef(v);
        }
        __syncthreads();
        if (l >= Lo) continue;
        for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < z.n; r += (int64_t)gridDim.x * blockDim.y) {
            typename V::Acc acc[PANEL_G];
            for (int t = 0; t < cnt; ++t) {
                const char* sl = static_cast<const char*>(z.panel) + t * slot_stride;
                const typename V::E q1 = V::ld(sl, r, l, L);
                const typename V::E q2 = MODE == 2 ? V::ld(sl, r, z.Lorig + l, L) : q1;
                const Coef* c = cs + (size_t)t * g * Lo + l;
#pragma unroll
                for (int k = 0; k < PANEL_G; ++k)
                    if (k < g) acc[k].add(c[(size_t)k * Lo], (MODE == 2 && c0 + k >= 2) ? q2 : q1);
            }
            if (MODE == 0) {
                double* srow = S + r * lds + l;
#pragma unroll
                for (int k = 0; k < PANEL_G; ++k)
                    if (k < g) srow[(size_t)(c0 + k) * L] += acc[k].value();
            } else if (MODE == 1) {
                double2* yr = z.Yacc + (size_t)r * z.Jtot * z.Lorig + l;
#pragma unroll
                for (int k = 0; k < PANEL_G; k += 2) {
                    if (k < g) {
                        double2* y = yr + (size_t)((c0 + k) >> 1) * z.Lorig;
                        double2 v = *y;
                        v.x += acc[k].value();
                        v.y += acc[k + 1].value();
                        *y = v;
                    }
                }
            } else {
                double2* y = z.Yacc + ((size_t)r * z.Jtot + z.jsel) * z.Lorig + l;
                double2 v = *y;
                v.x += acc[0].value() - acc[3].value();   // y1.re q1 - y2.im q2
                v.y += acc[1].value() + acc[2].value();   // y1.im q1 + y2.re q2
                *y = v;
            }
        }
    }
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) last = (atomicAdd(z.ctrl + C_TICKET3, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (last && threadIdx.x == 0 && threadIdx.y == 0) {
        z.ctrl[C_TICKET3] = 0;
        z.ctrl[C_PANEL] = i1;
    }
}

// R_j = X - (s_j I - H) Y_j (FP64), written as real blocks Rall[j] = [Re R_j | Im R_j]
// (n x 2L), and per (j, l) partial sums of |R_j|^2 over row chunks (blockIdx.x).
// HY is H Y with Y viewed as a real n x 2JL block.
__global__ void k_residual(const double2* __restrict__ Y, const double2* __restrict__ HY, const double* __restrict__ X,
                           int64_t ldx, const double2* __restrict__ quad, int64_t n, int J, int L,
                           double* __restrict__ Rall, double* __restrict__ part) {
    const int jl = blockIdx.y * blockDim.x + threadIdx.x;
    if (jl >= J * L) return;
    const int j = jl / L, l = jl % L;
    const double2 sj = quad[3 * j];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = r0 + chunk < n ? r0 + chunk : n;
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
        const double2 y = Y[(size_t)r * J * L + jl];
        const double2 hy = HY[(size_t)r * J * L + jl];
        const double x = X[r * ldx + l];
        const double re = x - (sj.x * y.x - sj.y * y.y) + hy.x;
        const double im = -(sj.x * y.y + sj.y * y.x) + hy.y;
        Rall[((size_t)j * n + r) * 2 * L + l] = re;
        Rall[((size_t)j * n + r) * 2 * L + L + l] = im;
        acc = __fma_rn(re, re, __fma_rn(im, im, acc));
    }
    part[(size_t)blockIdx.x * J * L + jl] = acc;
}

// max over (j, l) of ||R_j[:, l]|| / ||X[:, l]||, partials summed in chunk order
__global__ void k_residual_max(const double* __restrict__ part, int nchunks, int JL, int L, const double* __restrict__ xnorm,
                               double* __restrict__ out) {
    __shared__ double sh[256];
    double mx = 0.0;
    for (int jl = threadIdx.x; jl < JL; jl += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * JL + jl];
        const double xn = xnorm[jl % L];
        mx = fmax(mx, xn > 0.0 ? sqrt(s) / xn : 0.0);
    }
    sh[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// S[r][m L + l] = 2 Re sum_j w_j scaled_j^m Y[r][j][l], m < Mk
__global__ void k_moments_from_Y(const double2* __restrict__ Y, const double2* __restrict__ quad, int64_t n, int J, int L,
                                 int Mk, double* __restrict__ S, int64_t lds) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * L; e += stride) {
        const int64_t r = e / L;
        const int l = (int)(e % L);
        double* srow = S + r * lds + l;
        for (int m = 0; m < Mk; ++m) srow[(size_t)m * L] = 0.0;
        for (int j = 0; j < J; ++j) {
            const double2 y = Y[((size_t)r * J + j) * L + l];
            double2 f = quad[3 * j + 1];
            const double2 sc = quad[3 * j + 2];
            for (int m = 0; m < Mk; ++m) {
                srow[(size_t)m * L] += 2.0 * (f.x * y.x - f.y * y.y);
                f = cmul(f, sc);
            }
        }
    }
}

__global__ void k_zero_cols(double* S, int64_t n, int cols, int64_t lds) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * cols; e += stride)
        S[(e / cols) * lds + (e % cols)] = 0.0;
}

// Largest eigenvalue of T_K (alpha, beta of Lanczos column 0) by Sturm-count
// multisection: each of the 128 threads counts the eigenvalues below its own
// abscissa, and the bracket shrinks 129-fold per round.
__global__ void k_tri_maxeig(Lz z, double* out) {
    __shared__ double lo, hi;
    __shared__ int cnt[128];
    const int t = threadIdx.x, K = z.Kcol[0], L = z.L;
    if (K <= 0) { if (t == 0) *out = 0.0; return; }
    if (t == 0) {
        double l0 = 1e300, h0 = -1e300;
        for (int i = 0; i < K; ++i) {
            const double a = z.alpha[(size_t)i * L];
            const double r = (i > 0 ? fabs(z.beta[(size_t)i * L]) : 0.0) + (i + 1 < K ? fabs(z.beta[(size_t)(i + 1) * L]) : 0.0);
            l0 = fmin(l0, a - r);
            h0 = fmax(h0, a + r);
        }
        lo = l0;
        hi = h0;
    }
    __syncthreads();
    for (int round = 0; round < 8; ++round) {
        const double x = lo + (hi - lo) * (t + 1) / 129.0;
        int c = 0;
        double q = 1.0;
        for (int i = 0; i < K; ++i) {
            const double a = z.alpha[(size_t)i * L];
            const double b = i > 0 ? z.beta[(size_t)i * L] : 0.0;
            q = (a - x) - (i > 0 ? b * b / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++c;
        }
        cnt[t] = c;
        __syncthreads();
        if (t == 0) {
            // largest eigenvalue lies above the last abscissa with count < K
            int k = -1;
            for (int u = 0; u < 128; ++u) if (cnt[u] < K) k = u;
            const double w = (hi - lo) / 129.0;
            const double nlo = lo + w * (k + 1), nhi = lo + w * (k + 2);
            lo = nlo;
            hi = k == 127 ? hi : nhi;
        }
        __syncthreads();
    }
    if (t == 0) *out = hi;
}

// ----------------------------------------------------------------------------- host side
static int lz_grid(int64_t n, int L, int sm_count) {
    int by = 256 / L;
    if (by < 1) by = 1;
    int64_t g = (n + by - 1) / by;
    int cap = sm_count * 4;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// Panel length: as many steps as fit 96 KB of staged coefficients (a group of up to
// PANEL_G coefficient rows, 8 bytes each, for Lo output columns), a multiple of 3 (the
// three work vectors rotate every step) between 3 and 24.
static int panel_len(int kc, int Lo) {
    const int g = kc < PANEL_G ? kc : PANEL_G;
    int P = (int)((96 * 1024) / ((size_t)(g > 0 ? g : 1) * Lo * 8));
    if (P > 24) P = 24;
    P = P / 3 * 3;
    return P < 3 ? 3 : P;
}
static size_t panel_smem(int kc, int Lo, int P) {
    const int g = kc < PANEL_G ? kc : PANEL_G;
    return (size_t)P * g * Lo * 8;
}

// mode: the pass-2 output this state will serve (0 moments, 1 explicit solutions, 2 correction)
static void lz_alloc(Lz& z, Arena& ws, int64_t m, int64_t n, int L, int J, int Mk, int max_iter, int sm_count,
                     int mode) {
    z.n = n; z.L = L; z.J = J; z.Mk = Mk; z.max_iter = max_iter;
    for (int b = 0; b < 3; ++b) z.Q[b] = ws.take<double>((size_t)n * L);
    z.U = ws.take<double>((size_t)m * L);
    z.alpha = ws.take<double>((size_t)max_iter * L);
    z.beta = ws.take<double>((size_t)(max_iter + 1) * L);
    z.dcur = ws.take<double2>((size_t)(J > 0 ? J : 1) * L);
    z.tcur = ws.take<double2>((size_t)(J > 0 ? J : 1) * L);
    z.Dbuf = ws.take<double2>((size_t)max_iter * (J > 0 ? J : 1) * L);
    z.Ybuf = ws.take<double2>((size_t)max_iter * (J > 0 ? J : 1) * L);
    z.C = ws.take<double>((size_t)max_iter * (Mk > 0 ? Mk : 1) * L);
    z.Kcol = ws.take<int>(L);
    z.active = ws.take<int>(L);
    z.ctrl = ws.take<int>(C_WORDS);
    z.nblk = lz_grid(n, L, sm_count);
    z.partials = ws.take<double>((size_t)z.nblk * L);
    if (mode >= 0) {
        const int kc = mode == 0 ? Mk : (mode == 1 ? 2 * J : 4);
        z.P = panel_len(kc, mode == 2 ? L / 2 : L);
        z.panel = ws.take<double>((size_t)z.P * n * L);
    }
}

struct RefineBufs {
    double2* Y = nullptr;      // [n][J][L]
    double2* HY = nullptr;     // [n][J][L] (H applied to Y as a real n x 2JL block)
    double* U = nullptr;       // m x 2JL
    double* R = nullptr;       // [J][n][2L]
    double* part = nullptr;    // [nchunks][J L]
    double* xnorm = nullptr;   // [L]
    double* rmax = nullptr;    // [1]
    int nchunks = 0;
};

static void refine_alloc(RefineBufs& b, Lz& zc, Arena& ws, int64_t m, int64_t n, int L, int J, int max_iter, int sm) {
    b.Y = ws.take<double2>((size_t)n * J * L);
    b.HY = ws.take<double2>((size_t)n * J * L);
    b.U = ws.take<double>((size_t)m * 2 * J * L);
    b.R = ws.take<double>((size_t)J * n * 2 * L);
    b.nchunks = sm * 2;
    b.part = ws.take<double>((size_t)b.nchunks * J * L);
    b.xnorm = ws.take<double>(L);
    b.rmax = ws.take<double>(4);
    lz_alloc(zc, ws, m, n, 2 * L, 1, 0, max_iter, sm, 2);   // correction solves: 2L real columns, one shift
}

// Rounds of FP64 iterative refinement (params.refine; 0 = none, for either precision).
static int refine_rounds(const cmsvd_params* p) { return p->refine; }
// Tolerance of the recursive (Lanczos) residuals. In double-float the true residual sits a
// little above the recursive one (rounding at ~2^-48 instead of 2^-53); when the solves are
// checked in FP64 the mixed path iterates to a quarter of tol_solve, so that the check rarely
// needs a correction round.
static double inner_tol(const cmsvd_params* p) {
    return (p->precision == CMSVD_MIXED && p->refine > 0) ? 0.25 * p->tol_solve : p->tol_solve;
}

size_t krylov_workspace(const cmsvd_matrix* A, const cmsvd_params* p) {
    Arena a;
    Lz z;
    const bool refine = refine_rounds(p) > 0;
    lz_alloc(z, a, A->A.m, A->A.n, p->L, p->N / 2, p->M + 1, p->max_iter, A->ctx->sm_count, refine ? 1 : 0);
    a.take<double>((size_t)A->A.n * p->L);   // ell > 1 restart blocks (ping-pong)
    a.take<double>((size_t)A->A.n * p->L);
    if (refine) {
        RefineBufs b;
        Lz zc;
        refine_alloc(b, zc, a, A->A.m, A->A.n, p->L, p->N / 2, p->max_iter, A->ctx->sm_count);
    }
    return a.off + 256;
}

template <class V>
static int spmm_v(const Csr& A, int L, const void* X, void* Y, cudaStream_t s) {
    if (V::kind == SPMM_KIND_F64) return spmm(A, L, (const double*)X, L, (double*)Y, L, s);
    return spmm_df(A, L, (const float*)X, 2 * L, (float*)Y, 2 * L, s);
}

template <class V, int MODE>
static int launch_panel(Lz& z, double* S, int64_t lds, cudaStream_t s) {
    const int kc = MODE == 0 ? z.Mk : (MODE == 1 ? 2 * z.J : 4);
    const size_t smem = panel_smem(kc, MODE == 2 ? z.Lorig : z.L, z.P);
    // above 48 KB of shared memory in all (dynamic plus the kernel's static word) a launch needs the opt-in
    if (smem > 32 * 1024) CM_CUDA(cudaFuncSetAttribute(k_panel<V, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_panel<V, MODE><<<z.nblk, lz_block(z.L), smem, s>>>(z, S, lds);
    CM_LAUNCH();
    return CMSVD_OK;
}

// Pass 1 (+ pass 2 into S, or into z.Yacc for modes 1 and 2). Returns status; fills out.
template <class V>
static int lanczos_run(cmsvd_matrix* M, Lz& z, const double* X, int64_t ldx, double* S, int64_t lds,
                       int check_every, SolveOut* out) {
    void* Qb[3] = {z.Q[0], z.Q[1], z.Q[2]};
    cmsvd_context* ctx = M->ctx;
    cudaStream_t s = ctx->s;
    const dim3 blk = lz_block(z.L);
    const size_t shb = sizeof(double) * blk.x * blk.y;
    const int grid = z.nblk;
    if (V::kind == SPMM_KIND_DF) CM_TRY(csr_make_fp32(M));
    CM_CUDA(cudaMemsetAsync(z.ctrl, 0, sizeof(int) * C_WORDS, s));
    k_lz_norm0<<<grid, blk, shb, s>>>(z, X, ldx);
    CM_LAUNCH();
    k_lz_scale0<V><<<grid, blk, 0, s>>>(z, X, ldx, Qb[0]);
    CM_LAUNCH();
    // the SpMM autotuner runs here, outside the graph capture, on the real operands
    CM_TRY(spmm_tune(M->A, V::kind, z.L, Qb[0], V::kind == SPMM_KIND_F64 ? z.L : 2 * z.L, z.U,
                     V::kind == SPMM_KIND_F64 ? z.L : 2 * z.L, s));
    CM_TRY(spmm_tune(M->At, V::kind, z.L, z.U, V::kind == SPMM_KIND_F64 ? z.L : 2 * z.L, Qb[1],
                     V::kind == SPMM_KIND_F64 ? z.L : 2 * z.L, s));

    // ---- pass 1 as a graph of `chunk` iterations (a multiple of 3: buffer roles rotate)
    int chunk = ((check_every > 0 ? check_every : 48) + 2) / 3 * 3;
    if (chunk > 3 * ((z.max_iter + 2) / 3)) chunk = 3 * ((z.max_iter + 2) / 3);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    Profiler& pr = prof();
    pr.captured = 0;
    pr.capture_depth++;
    CM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < chunk; ++it) {
        const int p = it % 3;
        void* Qk = Qb[p];
        void* Qp = Qb[(p + 2) % 3];
        void* W = Qb[(p + 1) % 3];
        spmm_v<V>(M->A, z.L, Qk, z.U, s);
        spmm_v<V>(M->At, z.L, z.U, W, s);
        k_lz_dot<V><<<grid, blk, shb, s>>>(z, Qk, Qp, W);
        note_launch();
        k_lz_update<V><<<grid, blk, shb, s>>>(z, Qk, W);
        note_launch();
        k_lz_scale<V><<<grid, blk, 0, s>>>(z, W);
        note_launch();
    }
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    pr.capture_depth--;
    const int64_t nodes1 = pr.captured;
    if (ce != cudaSuccess) return cuda_fail(ce, "capture pass 1", __FILE__, __LINE__);
    ce = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "instantiate pass 1", __FILE__, __LINE__);
    int* h = ctx->pinned;
    int st = CMSVD_OK;
    // compulsory traffic per Lanczos step: A and A^T once each, X read and Y written by both
    // SpMMs, and the vector kernels (dot 4, update 3, scale 2 passes of n x L elements)
    const double nnz = (double)M->A.nnz, mm = (double)M->A.m, nn = (double)M->A.n, LL = z.L;
    const double ea = V::kind == SPMM_KIND_F64 ? 12.0
                      : (M->A.f32_exact == 0 ? 12.0 : (M->A.storage == CMSVD_STORE_BF16 ? 6.0 : 8.0));
    const double step_bytes = 2 * (ea * nnz) + 8.0 * (mm + nn + 2) + 2 * 8.0 * LL * (mm + nn) + 9 * 8.0 * nn * LL;
    const double step_flops = 4.0 * nnz * LL + 10.0 * nn * LL;
    for (;;) {
        ProfScope ps(CMSVD_PROF_KRYLOV, s, step_bytes * chunk, step_flops * chunk, nodes1);
        pr.launches += nodes1;
        ce = cudaGraphLaunch(ge, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(h, z.ctrl, sizeof(int) * C_WORDS, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { st = cuda_fail(ce, "pass 1", __FILE__, __LINE__); break; }
        if (h[C_NACT] == 0) break;
    }
    cudaGraphExecDestroy(ge);
    if (st != CMSVD_OK) return st;
    const int iters = h[C_IT];
    const int Kmax = h[C_KMAX];
    out->iters = iters;
    out->converged = (h[C_STATUS] & ST_NOTCONV) ? 0 : 1;
    out->breakdown = (h[C_STATUS] & ST_BREAKDOWN) ? 1 : 0;
    if (out->breakdown) return CMSVD_OK;
    if (S == nullptr && z.mode == 0) return CMSVD_OK;

    // ---- tridiagonal solves and moment coefficients
    if (z.mode == 0) {
        k_zero_cols<<<ctx->sm_count * 4, 256, 0, s>>>(S, z.n, z.L * z.Mk, lds);
        CM_LAUNCH();
    }
    if (Kmax == 0) return CMSVD_OK;
    k_tri_solve<<<(z.J * z.L + 127) / 128, 128, 0, s>>>(z);
    CM_LAUNCH();
    if (z.mode == 0) {
        k_tri_coef<<<(int)(((int64_t)Kmax * z.L + 255) / 256), 256, 0, s>>>(z, Kmax);
        CM_LAUNCH();
    }

    // ---- pass 2: chunks of P steps, each followed by its panel fold
    k_lz_scale0<V><<<grid, blk, 0, s>>>(z, X, ldx, Qb[0]);
    CM_LAUNCH();
    const int chunk2 = z.P;
    pr.captured = 0;
    pr.capture_depth++;
    CM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < chunk2; ++it) {
        const int p = it % 3;
        void* Qk = Qb[p];
        void* Qp = Qb[(p + 2) % 3];
        void* W = Qb[(p + 1) % 3];
        spmm_v<V>(M->A, z.L, Qk, z.U, s);
        spmm_v<V>(M->At, z.L, z.U, W, s);
        k_lz2_step<V><<<grid, blk, 0, s>>>(z, Qk, Qp, W);
        note_launch();
    }
    int pst = z.mode == 0 ? launch_panel<V, 0>(z, S, lds, s)
                          : (z.mode == 1 ? launch_panel<V, 1>(z, S, lds, s) : launch_panel<V, 2>(z, S, lds, s));
    ce = cudaStreamEndCapture(s, &g);
    pr.capture_depth--;
    const int64_t nodes2 = pr.captured;
    if (pst != CMSVD_OK) { if (ce == cudaSuccess) cudaGraphDestroy(g); return pst; }
    if (ce != cudaSuccess) return cuda_fail(ce, "capture pass 2", __FILE__, __LINE__);
    ce = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "instantiate pass 2", __FILE__, __LINE__);
    const int kc = z.mode == 0 ? z.Mk : (z.mode == 1 ? 2 * z.J : 4);
    const double step2_bytes = 2 * (ea * nnz) + 8.0 * (mm + nn + 2) + 2 * 8.0 * LL * (mm + nn) + 6 * 8.0 * nn * LL +
                               (z.mode == 0 ? 16.0 * nn * LL * z.Mk : 32.0 * nn * LL * z.J) / z.P;
    const double step2_flops = 4.0 * nnz * LL + nn * LL * (6.0 + 2.0 * kc);
    for (int done = 0; done < Kmax; done += chunk2) {
        ProfScope ps(CMSVD_PROF_KRYLOV, s, step2_bytes * chunk2, step2_flops * chunk2, nodes2);
        pr.launches += nodes2;
        ce = cudaGraphLaunch(ge, s);
        if (ce != cudaSuccess) break;
    }
    cudaGraphExecDestroy(ge);
    if (ce != cudaSuccess) return cuda_fail(ce, "pass 2", __FILE__, __LINE__);
    return CMSVD_OK;
}

// One filter application with FP64 iterative refinement: explicit Y_j from the shared
// Lanczos process, then rounds of R_j = X - (s_j I - H) Y_j, computed in FP64 with FP64 A,
// and corrections (s_j I - H) E_j = R_j (one Lanczos run per shift on [Re R_j | Im R_j])
// until max ||R_j|| / ||X|| <= tol_solve or the round limit; finally the Mk moments.
template <class V>
static int refined_filter(cmsvd_matrix* M, const cmsvd_params* p, Lz& z, Lz& zc, RefineBufs& rb, const double* X,
                          int64_t ldx, int Mk, double* S, int64_t lds, SolveOut* out) {
    cmsvd_context* ctx = M->ctx;
    cudaStream_t s = ctx->s;
    const int J = z.J, L = z.L;
    const int64_t n = z.n;
    CM_CUDA(cudaMemsetAsync(rb.Y, 0, sizeof(double2) * n * J * L, s));
    z.mode = 1;
    z.Yacc = rb.Y;
    z.Jtot = J;
    z.Lorig = L;
    CM_TRY(lanczos_run<V>(M, z, X, ldx, nullptr, 0, p->check_every, out));
    z.mode = 0;
    if (out->breakdown) { set_error("Lanczos breakdown (non-finite value)"); return CMSVD_BREAKDOWN; }
    CM_CUDA(cudaMemcpyAsync(rb.xnorm, z.beta, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    int64_t iters = out->iters;
    int rounds = 0;
    int max_rounds = refine_rounds(p);
    bool inner_v = V::kind != SPMM_KIND_F64;   // corrections in the solve's own format until they stop helping
    bool stagnated = false;
    double rmax = 0.0, rprev = 0.0;
    for (;;) {
        // H Y in FP64 (Y as a real n x 2JL block)
        CM_TRY(spmm(M->A, 2 * J * L, (const double*)rb.Y, 2 * J * L, rb.U, 2 * J * L, s));
        CM_TRY(spmm(M->At, 2 * J * L, rb.U, 2 * J * L, (double*)rb.HY, 2 * J * L, s));
        {
            ProfScope ps(CMSVD_PROF_OTHER, s, 8.0 * n * (4.0 * J * L + L) + 16.0 * J * n * L, 10.0 * n * J * L, 2);
            dim3 grid(rb.nchunks, (J * L + 127) / 128);
            k_residual<<<grid, 128, 0, s>>>(rb.Y, rb.HY, X, ldx, z.quad, n, J, L, rb.R, rb.part);
            CM_LAUNCH();
            k_residual_max<<<1, 256, 0, s>>>(rb.part, rb.nchunks, J * L, L, rb.xnorm, rb.rmax);
            CM_LAUNCH();
        }
        CM_CUDA(cudaMemcpyAsync(ctx->pinned, rb.rmax, sizeof(double), cudaMemcpyDeviceToHost, s));
        CM_CUDA(cudaStreamSynchronize(s));
        memcpy(&rmax, ctx->pinned, sizeof(double));
        if (!(rmax == rmax)) { set_error("refinement residual is not finite"); return CMSVD_BREAKDOWN; }
        // Stop at the tolerance or the round limit. When the residual no longer halves: with
        // double-float corrections, switch them to FP64; with FP64 corrections the residual has
        // reached the rounding floor of its own FP64 evaluation, ~u ||A^T A|| ||Y_j||, and the
        // solves are as accurate as FP64 allows.
        if (rmax <= p->tol_solve || rounds >= max_rounds) break;
        if (rounds > 0 && rmax > 0.5 * rprev) {
            if (!inner_v) { stagnated = true; break; }
            inner_v = false;
            max_rounds = rounds + (p->refine > 0 ? p->refine : 2);
        }
        rprev = rmax;
        ++rounds;
        for (int j = 0; j < J; ++j) {
            zc.quad = z.quad + 3 * j;
            zc.mode = 2;
            zc.Yacc = rb.Y;
            zc.Jtot = J;
            zc.Lorig = L;
            zc.jsel = j;
            zc.tol = p->tol_solve;
            zc.fault_at = 0;
            SolveOut so;
            if (inner_v) CM_TRY(lanczos_run<V>(M, zc, rb.R + (size_t)j * n * 2 * L, 2 * L, nullptr, 0, p->check_every, &so));
            else CM_TRY(lanczos_run<VecF64>(M, zc, rb.R + (size_t)j * n * 2 * L, 2 * L, nullptr, 0, p->check_every, &so));
            if (so.breakdown) { set_error("Lanczos breakdown in a correction solve"); return CMSVD_BREAKDOWN; }
            iters += so.iters;
            if (!so.converged) out->converged = 0;
        }
    }
    out->iters = iters;
    out->refine_rounds = rounds;
    out->refine_residual = rmax;
    // converged: the tolerance was met, or FP64 corrections reached the FP64 rounding floor
    if (!(rmax <= p->tol_solve) && !stagnated) out->converged = 0;
    {
        ProfScope ps(CMSVD_PROF_OTHER, s, 16.0 * n * J * L + 8.0 * n * L * Mk, 4.0 * n * J * L * Mk);
        k_moments_from_Y<<<ctx->sm_count * 4, 256, 0, s>>>(rb.Y, z.quad, n, J, L, Mk, S, lds);
        CM_LAUNCH();
    }
    return CMSVD_OK;
}

template <class V>
static int filter_moments(cmsvd_matrix* M, const cmsvd_params* p, Lz& z, Lz& zc, RefineBufs& rb, bool use_refine,
                          double** Xr, const double* X, int64_t ldx, int Mk, double* S, int64_t lds, SolveOut* out) {
    const double* Xc = X;
    int64_t ldc = ldx;
    // iteration technique (Eq. iter1): S_0^(nu) = 2 Re sum_j w_j (s_j I - H)^{-1} S_0^(nu-1)
    for (int nu = 1; nu < p->ell; ++nu) {
        z.Mk = 1;
        double* dst = Xr[nu & 1];
        if (use_refine) {
            CM_TRY(refined_filter<V>(M, p, z, zc, rb, Xc, ldc, 1, dst, p->L, out));
        } else {
            CM_TRY(lanczos_run<V>(M, z, Xc, ldc, dst, p->L, p->check_every, out));
            if (out->breakdown) { set_error("Lanczos breakdown (non-finite value)"); return CMSVD_BREAKDOWN; }
        }
        Xc = dst;
        ldc = p->L;
    }
    z.Mk = Mk;
    if (use_refine) return refined_filter<V>(M, p, z, zc, rb, Xc, ldc, Mk, S, lds, out);
    CM_TRY(lanczos_run<V>(M, z, Xc, ldc, S, lds, p->check_every, out));
    if (out->breakdown) { set_error("Lanczos breakdown (non-finite value)"); return CMSVD_BREAKDOWN; }
    return CMSVD_OK;
}

int krylov_moments(cmsvd_matrix* M, const cmsvd_params* p, const double2* quad, int Mk, const double* X,
                   int64_t ldx, double* S, int64_t lds, Arena& ws, SolveOut* out) {
    cmsvd_context* ctx = M->ctx;
    const bool use_refine = refine_rounds(p) > 0;
    Lz z;
    lz_alloc(z, ws, M->A.m, M->A.n, p->L, p->N / 2, p->M + 1, p->max_iter, ctx->sm_count, use_refine ? 1 : 0);
    double* Xr[2] = {ws.take<double>((size_t)M->A.n * p->L), ws.take<double>((size_t)M->A.n * p->L)};
    RefineBufs rb;
    Lz zc;
    if (use_refine) refine_alloc(rb, zc, ws, M->A.m, M->A.n, p->L, p->N / 2, p->max_iter, ctx->sm_count);
    if (!ws.fits()) { set_error("workspace too small"); return CMSVD_WORKSPACE_TOO_SMALL; }
    z.tol = inner_tol(p);
    z.quad = quad;
    z.fault_at = p->fault_breakdown_at;
    if (p->precision == CMSVD_MIXED) return filter_moments<VecDF>(M, p, z, zc, rb, use_refine, Xr, X, ldx, Mk, S, lds, out);
    return filter_moments<VecF64>(M, p, z, zc, rb, use_refine, Xr, X, ldx, Mk, S, lds, out);
}

// ||A||_2 by 128 Lanczos steps on H from a fixed deterministic start vector.
__global__ void k_fill_start(double* x, int64_t n) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        x[i] = 1.0 + 0.5 * sin(0.7 * (double)i);
}

int norm_estimate(cmsvd_matrix* M, Arena& ws, double* norm_out) {
    cmsvd_context* ctx = M->ctx;
    Lz z;
    int steps = (int)(M->A.n < 128 ? M->A.n : 128);
    lz_alloc(z, ws, M->A.m, M->A.n, 1, 0, 0, steps, ctx->sm_count, -1);
    double* x = ws.take<double>(M->A.n);
    double* lam = ws.take<double>(1);
    if (!ws.fits()) { set_error("workspace too small"); return CMSVD_WORKSPACE_TOO_SMALL; }
    z.tol = -1.0;
    k_fill_start<<<ctx->sm_count, 256, 0, ctx->s>>>(x, M->A.n);
    CM_LAUNCH();
    SolveOut so;
    CM_TRY(lanczos_run<VecF64>(M, z, x, 1, nullptr, 0, 48, &so));
    k_tri_maxeig<<<1, 128, 0, ctx->s>>>(z, lam);
    CM_LAUNCH();
    CM_CUDA(cudaMemcpyAsync(ctx->pinned, lam, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CM_CUDA(cudaStreamSynchronize(ctx->s));
    double hv;
    memcpy(&hv, ctx->pinned, sizeof(double));
    *norm_out = sqrt(hv > 0 ? hv : 0.0);
    return CMSVD_OK;
}

}  // namespace cmsvd
