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
//           explicitly rounded operations) and accumulate S_k += c_{k,i} q_i.
// The SpMM is real (L columns), not complex (2L). Iterations run as CUDA
// graphs; convergence is polled every check_every iterations.
// With precision MIXED the Lanczos vectors, the SpMM values and its accumulation are
// FP32 (alpha, beta, the LDL^T recurrences and S stay FP64), and every shifted solve is
// refined in FP64 (refined_filter, at the end of this file).
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

// explicitly rounded operations of the vector recurrences (FP64 or FP32 vectors):
// pass 2 repeats pass 1's operations exactly, so the regenerated vectors are bitwise equal
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double div_t(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_t(float a, float b) { return __fdiv_rn(a, b); }

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

// ----------------------------------------------------------------------------- Lanczos state
enum { C_IT = 0, C_NACT = 1, C_STATUS = 2, C_TICKET = 3, C_IT2 = 4, C_KMAX = 5, C_TICKET2 = 6, C_WORDS = 8 };
enum { ST_BREAKDOWN = 1, ST_NOTCONV = 2 };

struct Lz {
    int64_t n = 0;
    int L = 0, J = 0, Mk = 0, max_iter = 0;
    double tol = 0.0;          // < 0: never converge (norm estimation)
    double* Q[3] = {nullptr, nullptr, nullptr};
    double* U = nullptr;       // m x L
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
    // pass-2 accumulation of explicit solutions (refinement): 0 = moments into S,
    // 1 = Yacc[r][j][l] += y_{i,j,l} q_i (all shifts), 2 = correction for shift jsel:
    // columns l and Lorig + l carry Re and Im of the right-hand side,
    // Yacc[r][jsel][l] += y_l q_l + i y_{Lorig+l} q_{Lorig+l}.
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

template <typename T>
__global__ void k_lz_scale0(Lz z, const double* __restrict__ X, int64_t ldx, T* __restrict__ Q0) {
    const int l = threadIdx.x;
    const double b = z.beta[l];
    const bool act = b > 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < z.n; i += (int64_t)gridDim.x * blockDim.y)
        Q0[i * z.L + l] = act ? (T)__ddiv_rn(X[i * ldx + l], b) : (T)0;
}

// pass 1, part 1: w <- H q_k - beta_k q_{k-1};  alpha_k = q_k^T w
template <typename T>
__global__ void k_lz_dot(Lz z, const T* __restrict__ Qk, const T* __restrict__ Qp, T* __restrict__ W) {
    extern __shared__ double sh[];
    if (z.ctrl[C_NACT] == 0) return;
    const int k = z.ctrl[C_IT];
    const int l = threadIdx.x;
    const bool act = z.active[l] != 0;
    const T b = (T)(k > 0 ? z.beta[(size_t)k * z.L + l] : 0.0);
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < z.n; i += (int64_t)gridDim.x * blockDim.y) {
        const int64_t o = i * z.L + l;
        T w = (T)0;
        if (act) {
            w = W[o];
            if (k > 0) w = fma_t(-b, Qp[o], w);
            acc = __fma_rn((double)Qk[o], (double)w, acc);
        }
        W[o] = w;
    }
    if (column_reduce(acc, sh, z.partials, z.ctrl + C_TICKET, z.L)) {
        if (threadIdx.y == 0) z.alpha[(size_t)k * z.L + l] = act ? sh[l] : 0.0;
    }
}

// pass 1, part 2: w <- w - alpha_k q_k;  beta_{k+1} = ||w||; per (shift, column)
// LDL^T pivot d and t = e_k^T (s I - T_k)^{-1} e_1 beta_1; convergence and freezing.
template <typename T>
__global__ void k_lz_update(Lz z, const T* __restrict__ Qk, T* __restrict__ W) {
    extern __shared__ double sh[];
    if (z.ctrl[C_NACT] == 0) return;
    const int k = z.ctrl[C_IT];
    const int l = threadIdx.x;
    const bool act = z.active[l] != 0;
    const double a = z.alpha[(size_t)k * z.L + l];
    const T at = (T)a;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < z.n; i += (int64_t)gridDim.x * blockDim.y) {
        const int64_t o = i * z.L + l;
        if (act) {
            const T w = fma_t(-at, Qk[o], W[o]);
            W[o] = w;
            acc = __fma_rn((double)w, (double)w, acc);
        }
    }
    if (!column_reduce(acc, sh, z.partials, z.ctrl + C_TICKET, z.L)) return;
    if (threadIdx.y == 0) {
        const double bnext = sqrt(sh[l]);
        if (!act) {
            z.beta[(size_t)(k + 1) * z.L + l] = 0.0;
        } else {
            z.beta[(size_t)(k + 1) * z.L + l] = bnext;
            const double b1 = z.beta[l];
            const double bk = z.beta[(size_t)k * z.L + l];
            bool allconv = z.J > 0 && z.tol >= 0.0;
            bool bad = !isfinite(bnext) || !isfinite(a);
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
template <typename T>
__global__ void k_lz_scale(Lz z, T* __restrict__ W) {
    const int kk = z.ctrl[C_IT];   // already k+1
    const int l = threadIdx.x;
    const bool act = z.active[l] != 0;
    const T b = (T)(act ? z.beta[(size_t)kk * z.L + l] : 1.0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < z.n; i += (int64_t)gridDim.x * blockDim.y) {
        const int64_t o = i * z.L + l;
        W[o] = act ? div_t(W[o], b) : (T)0;
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

// pass 2: S_m += c_{m,i} q_i; then q_{i+1} from the stored alpha, beta with the
// same rounded operations as pass 1.
template <typename T>
__global__ void k_lz2_step(Lz z, const T* __restrict__ Qk, const T* __restrict__ Qp, T* __restrict__ W,
                           double* __restrict__ S, int64_t lds) {
    const int i = z.ctrl[C_IT2];
    if (i >= z.ctrl[C_KMAX]) return;
    const int l = threadIdx.x;
    const int K = z.Kcol[l];
    const bool live = i < K;
    const bool next = i + 1 < K;
    const double a = z.alpha[(size_t)i * z.L + l];
    const double b = i > 0 ? z.beta[(size_t)i * z.L + l] : 0.0;
    const double bn = next ? z.beta[(size_t)(i + 1) * z.L + l] : 1.0;
    const int Mk = z.Mk;
    const double* c = z.C + (size_t)i * Mk * z.L + l;
    const T at = (T)a, bt = (T)b, bnt = (T)bn;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < z.n; r += (int64_t)gridDim.x * blockDim.y) {
        const int64_t o = r * z.L + l;
        const T q = Qk[o];
        if (live) {
            double* srow = S + r * lds + l;
            for (int m = 0; m < Mk; ++m) srow[m * z.L] = __fma_rn(c[(size_t)m * z.L], (double)q, srow[m * z.L]);
        }
        T w = (T)0;
        if (next) {
            w = W[o];
            if (i > 0) w = fma_t(-bt, Qp[o], w);
            w = fma_t(-at, q, w);
            w = div_t(w, bnt);
        }
        W[o] = w;
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

// pass 2 with accumulation of explicit solutions (refinement modes 1 and 2)
template <typename T>
__global__ void k_lz2_step_acc(Lz z, const T* __restrict__ Qk, const T* __restrict__ Qp, T* __restrict__ W) {
    const int i = z.ctrl[C_IT2];
    if (i >= z.ctrl[C_KMAX]) return;
    const int l = threadIdx.x;
    const int K = z.Kcol[l];
    const bool live = i < K;
    const bool next = i + 1 < K;
    const double a = z.alpha[(size_t)i * z.L + l];
    const double b = i > 0 ? z.beta[(size_t)i * z.L + l] : 0.0;
    const double bn = next ? z.beta[(size_t)(i + 1) * z.L + l] : 1.0;
    const size_t JL = (size_t)z.J * z.L;
    // mode 2: the thread of column l < Lorig also owns column Lorig + l
    const int l2 = l + z.Lorig;
    const bool pair = z.mode == 2 && l < z.Lorig;
    const bool live2 = pair && i < z.Kcol[l2];
    double2 y1 = make_double2(0, 0), y2 = make_double2(0, 0);
    if (z.mode == 2) {
        if (pair && live) y1 = z.Ybuf[i * JL + l];
        if (live2) y2 = z.Ybuf[i * JL + l2];
    }
    const T at = (T)a, bt = (T)b, bnt = (T)bn;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < z.n; r += (int64_t)gridDim.x * blockDim.y) {
        const int64_t o = r * z.L + l;
        const T qt = Qk[o];
        const double q = (double)qt;
        if (z.mode == 1) {
            if (live) {
                double2* yr = z.Yacc + ((size_t)r * z.Jtot) * z.Lorig + l;
                for (int j = 0; j < z.J; ++j) {
                    const double2 c = z.Ybuf[i * JL + (size_t)j * z.L + l];
                    double2 v = yr[(size_t)j * z.Lorig];
                    v.x = __fma_rn(c.x, q, v.x);
                    v.y = __fma_rn(c.y, q, v.y);
                    yr[(size_t)j * z.Lorig] = v;
                }
            }
        } else if (pair && (live || live2)) {
            const double q2 = (double)Qk[r * z.L + l2];
            double2* yp = z.Yacc + ((size_t)r * z.Jtot + z.jsel) * z.Lorig + l;
            double2 v = *yp;
            // (y1 q) + i (y2 q2) = (y1.x q - y2.y q2) + i (y1.y q + y2.x q2)
            v.x = __fma_rn(y1.x, q, __fma_rn(-y2.y, q2, v.x));
            v.y = __fma_rn(y1.y, q, __fma_rn(y2.x, q2, v.y));
            *yp = v;
        }
        T w = (T)0;
        if (next) {
            w = W[o];
            if (i > 0) w = fma_t(-bt, Qp[o], w);
            w = fma_t(-at, qt, w);
            w = div_t(w, bnt);
        }
        W[o] = w;
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
    int cap = sm_count * 2;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

static void lz_alloc(Lz& z, Arena& ws, int64_t m, int64_t n, int L, int J, int Mk, int max_iter, int sm_count) {
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
    lz_alloc(zc, ws, m, n, 2 * L, 1, 0, max_iter, sm);   // correction solves: 2L real columns, one shift
}

size_t krylov_workspace(const cmsvd_matrix* A, const cmsvd_params* p) {
    Arena a;
    Lz z;
    lz_alloc(z, a, A->A.m, A->A.n, p->L, p->N / 2, p->M + 1, p->max_iter, A->ctx->sm_count);
    a.take<double>((size_t)A->A.n * p->L);   // ell > 1 restart blocks (ping-pong)
    a.take<double>((size_t)A->A.n * p->L);
    if (p->refine > 0 || p->precision == CMSVD_MIXED) {
        RefineBufs b;
        Lz zc;
        refine_alloc(b, zc, a, A->A.m, A->A.n, p->L, p->N / 2, p->max_iter, A->ctx->sm_count);
    }
    return a.off + 256;
}

// Pass 1 (+ optional pass 2 into S). Returns status; fills out.
template <typename T>
static int lanczos_run(cmsvd_matrix* M, Lz& z, const double* X, int64_t ldx, double* S, int64_t lds,
                       int check_every, SolveOut* out) {
    T* Qb[3] = {(T*)z.Q[0], (T*)z.Q[1], (T*)z.Q[2]};
    T* Ub = (T*)z.U;
    cmsvd_context* ctx = M->ctx;
    cudaStream_t s = ctx->s;
    const dim3 blk = lz_block(z.L);
    const size_t shb = sizeof(double) * blk.x * blk.y;
    const int grid = z.nblk;
    CM_CUDA(cudaMemsetAsync(z.ctrl, 0, sizeof(int) * C_WORDS, s));
    k_lz_norm0<<<grid, blk, shb, s>>>(z, X, ldx);
    CM_LAUNCH();
    k_lz_scale0<T><<<grid, blk, 0, s>>>(z, X, ldx, Qb[0]);
    CM_LAUNCH();

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
        T* Qk = Qb[p];
        T* Qp = Qb[(p + 2) % 3];
        T* W = Qb[(p + 1) % 3];
        spmm(M->A, z.L, Qk, z.L, Ub, z.L, s);
        spmm(M->At, z.L, Ub, z.L, W, z.L, s);
        k_lz_dot<T><<<grid, blk, shb, s>>>(z, Qk, Qp, W);
        k_lz_update<T><<<grid, blk, shb, s>>>(z, Qk, W);
        k_lz_scale<T><<<grid, blk, 0, s>>>(z, W);
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
    // compulsory traffic per Lanczos step: A and A^T once each, X read and Y written by
    // both SpMMs, and the vector kernels (dot 4, update 3, scale 2 n x L passes)
    const double nnz = (double)M->A.nnz, mm = (double)M->A.m, nn = (double)M->A.n, LL = z.L;
    const double eb = (double)sizeof(T), ea = sizeof(T) + 4.0;
    const double step_bytes = 2 * (ea * nnz) + 8.0 * (mm + nn + 2) + 2 * eb * LL * (mm + nn) + 9 * eb * nn * LL;
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
    if (S == nullptr && z.mode == 0) return CMSVD_OK;

    // ---- tridiagonal solves and moment coefficients
    CM_TRY(Kmax >= 0 ? CMSVD_OK : CMSVD_BREAKDOWN);
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

    // ---- pass 2
    k_lz_scale0<T><<<grid, blk, 0, s>>>(z, X, ldx, Qb[0]);
    CM_LAUNCH();
    int chunk2 = chunk;
    if (chunk2 > 3 * ((Kmax + 2) / 3)) chunk2 = 3 * ((Kmax + 2) / 3);
    pr.captured = 0;
    pr.capture_depth++;
    CM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < chunk2; ++it) {
        const int p = it % 3;
        T* Qk = Qb[p];
        T* Qp = Qb[(p + 2) % 3];
        T* W = Qb[(p + 1) % 3];
        spmm(M->A, z.L, Qk, z.L, Ub, z.L, s);
        spmm(M->At, z.L, Ub, z.L, W, z.L, s);
        if (z.mode == 0) k_lz2_step<T><<<grid, blk, 0, s>>>(z, Qk, Qp, W, S, lds);
        else k_lz2_step_acc<T><<<grid, blk, 0, s>>>(z, Qk, Qp, W);
    }
    ce = cudaStreamEndCapture(s, &g);
    pr.capture_depth--;
    const int64_t nodes2 = pr.captured;
    if (ce != cudaSuccess) return cuda_fail(ce, "capture pass 2", __FILE__, __LINE__);
    ce = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "instantiate pass 2", __FILE__, __LINE__);
    const double step2_bytes = 2 * (ea * nnz) + 8.0 * (mm + nn + 2) + 2 * eb * LL * (mm + nn) + 4 * eb * nn * LL +
                               (z.mode == 0 ? 16.0 * nn * LL * z.Mk : 32.0 * nn * LL * z.J);
    const double step2_flops = 4.0 * nnz * LL + nn * LL * (6.0 + 2.0 * z.Mk);
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

// Refinement rounds: the FP32 path always refines (default 8 rounds).
static int refine_rounds(const cmsvd_params* p) {
    if (p->precision == CMSVD_MIXED) return p->refine > 0 ? p->refine : 8;
    return p->refine;
}
// Tolerance of the inner (Lanczos) solves: FP32 vectors stop near their own accuracy.
static double inner_tol(const cmsvd_params* p) {
    return p->precision == CMSVD_MIXED ? fmax(p->tol_solve, 1e-6) : p->tol_solve;
}

// One filter application with FP64 iterative refinement: explicit Y_j from the shared
// Lanczos process, then rounds of R_j = X - (s_j I - H) Y_j and corrections
// (s_j I - H) E_j = R_j (one Lanczos run per shift on [Re R_j | Im R_j]) until
// max ||R_j|| / ||X|| <= tol_solve or p->refine rounds; finally the Mk moments.
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
    const bool mixed = p->precision == CMSVD_MIXED;
    if (mixed) CM_TRY(lanczos_run<float>(M, z, X, ldx, nullptr, 0, p->check_every, out));
    else CM_TRY(lanczos_run<double>(M, z, X, ldx, nullptr, 0, p->check_every, out));
    if (out->breakdown) { set_error("Lanczos breakdown (non-finite value)"); return CMSVD_BREAKDOWN; }
    CM_CUDA(cudaMemcpyAsync(rb.xnorm, z.beta, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    int64_t iters = out->iters;
    int rounds = 0;
    int max_rounds = refine_rounds(p);
    bool inner32 = mixed;   // correction solves in FP32 until they stop helping
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
        // FP32 corrections, switch them to FP64 (FP32 vectors cannot resolve shifts close to
        // the spectrum); with FP64 corrections the residual has reached the rounding floor of
        // its own FP64 evaluation, ~u ||A^T A|| ||Y_j||, and the solves are as accurate as FP64 allows.
        if (rmax <= p->tol_solve || rounds >= max_rounds) break;
        if (rounds > 0 && rmax > 0.5 * rprev) {
            if (!inner32) { stagnated = true; break; }
            inner32 = false;
            max_rounds = rounds + (p->refine > 0 ? p->refine : 4);
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
            zc.tol = inner32 ? inner_tol(p) : p->tol_solve;
            SolveOut so;
            if (inner32) CM_TRY(lanczos_run<float>(M, zc, rb.R + (size_t)j * n * 2 * L, 2 * L, nullptr, 0, p->check_every, &so));
            else CM_TRY(lanczos_run<double>(M, zc, rb.R + (size_t)j * n * 2 * L, 2 * L, nullptr, 0, p->check_every, &so));
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
    z.mode = 0;
    return CMSVD_OK;
}

int krylov_moments(cmsvd_matrix* M, const cmsvd_params* p, const double2* quad, int Mk, const double* X,
                   int64_t ldx, double* S, int64_t lds, Arena& ws, SolveOut* out) {
    cmsvd_context* ctx = M->ctx;
    Lz z;
    lz_alloc(z, ws, M->A.m, M->A.n, p->L, p->N / 2, p->M + 1, p->max_iter, ctx->sm_count);
    double* Xr[2] = {ws.take<double>((size_t)M->A.n * p->L), ws.take<double>((size_t)M->A.n * p->L)};
    RefineBufs rb;
    Lz zc;
    if (refine_rounds(p) > 0) refine_alloc(rb, zc, ws, M->A.m, M->A.n, p->L, p->N / 2, p->max_iter, ctx->sm_count);
    if (p->precision == CMSVD_MIXED) CM_TRY(csr_make_fp32(M));
    if (!ws.fits()) { set_error("workspace too small"); return CMSVD_WORKSPACE_TOO_SMALL; }
    z.tol = inner_tol(p);
    z.quad = quad;
    const bool use_refine = refine_rounds(p) > 0;
    const double* Xc = X;
    int64_t ldc = ldx;
    // iteration technique (Eq. iter1): S_0^(nu) = 2 Re sum_j w_j (s_j I - H)^{-1} S_0^(nu-1)
    for (int nu = 1; nu < p->ell; ++nu) {
        z.Mk = 1;
        double* dst = Xr[nu & 1];
        if (use_refine) {
            CM_TRY(refined_filter(M, p, z, zc, rb, Xc, ldc, 1, dst, p->L, out));
        } else {
            CM_TRY(lanczos_run<double>(M, z, Xc, ldc, dst, p->L, p->check_every, out));
            if (out->breakdown) { set_error("Lanczos breakdown (non-finite value)"); return CMSVD_BREAKDOWN; }
        }
        Xc = dst;
        ldc = p->L;
    }
    z.Mk = Mk;
    if (use_refine) return refined_filter(M, p, z, zc, rb, Xc, ldc, Mk, S, lds, out);
    CM_TRY(lanczos_run<double>(M, z, Xc, ldc, S, lds, p->check_every, out));
    if (out->breakdown) { set_error("Lanczos breakdown (non-finite value)"); return CMSVD_BREAKDOWN; }
    return CMSVD_OK;
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
    lz_alloc(z, ws, M->A.m, M->A.n, 1, 0, 0, steps, ctx->sm_count);
    double* x = ws.take<double>(M->A.n);
    double* lam = ws.take<double>(1);
    if (!ws.fits()) { set_error("workspace too small"); return CMSVD_WORKSPACE_TOO_SMALL; }
    z.tol = -1.0;
    k_fill_start<<<ctx->sm_count, 256, 0, ctx->s>>>(x, M->A.n);
    CM_LAUNCH();
    SolveOut so;
    CM_TRY(lanczos_run<double>(M, z, x, 1, nullptr, 0, 48, &so));
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
