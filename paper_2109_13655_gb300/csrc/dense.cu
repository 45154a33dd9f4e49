// Dense FP64 kernels of the Rayleigh-Ritz part (Alg. 1 steps 3-5):
//   - Gram G = X^T Y of tall-skinny blocks (deterministic split-n reduction),
//   - Z = X W for tall X and small W,
//   - Cholesky (one CTA, or a cooperative blocked form), triangular inverse,
//   - the orthogonalization X = Q R of the rank truncation of S^ (step 3): two shifted
//     CholeskyQR passes, deflation by a pivoted Cholesky, a congruence polish and one
//     pass from the data; and of qr(A V~) (step 4): one Cholesky of the Gram when its
//     rounding is provably negligible, else CholeskyQR2, else the deflated form,
//   - one-sided Jacobi SVD of a small square matrix (SVD of R in step 3 and of B
//     in step 5), which keeps the high relative accuracy of small singular values.
// FP64 on this part runs on the FP64 pipe (no FP64 tensor-core path is used).
#include "internal.cuh"
#include <mutex>

namespace cmsvd {

// ----------------------------------------------------------------------------- Gram
constexpr int GT = 64;   // output tile
constexpr int GK = 16;   // rows per slab

__global__ void __launch_bounds__(256, 4) k_gram_partial(const double* __restrict__ X, int64_t ldx, int c1,
                                                      const double* __restrict__ Y, int64_t ldy, int c2, int64_t n,
                                                      int64_t rows_per_chunk, int sym, double* __restrict__ partials) {
    __shared__ double Xs[GK][GT];
    __shared__ double Ys[GK][GT];
    const int ti = blockIdx.x * GT, tj = blockIdx.y * GT;
    if (sym && blockIdx.x > blockIdx.y) return;   // symmetric: lower tiles are mirrored by the sum
    const int64_t r0 = (int64_t)blockIdx.z * rows_per_chunk;
    const int64_t r1 = r0 + rows_per_chunk < n ? r0 + rows_per_chunk : n;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    if (sym && blockIdx.x == blockIdx.y) {
        // Diagonal tile of a symmetric Gram: only its 136 upper 4 x 4 blocks are computed,
        // one per thread in row-major order of the upper triangle, so warps 5-7 skip the
        // multiply-adds (GB300 charges an FP64 warp instruction whatever its active lanes).
        // The lower entries are mirrored when the partials are summed. Every computed entry
        // runs the same multiply-adds in the same order as in the general path.
        const bool active = tid < 136;
        int by = 0, rem = tid;
        if (active)
            while (rem >= 16 - by) { rem -= 16 - by; ++by; }
        const int bx = by + rem;
        for (int64_t r = r0; r < r1; r += GK) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = tid + 256 * q, rr = e / GT, cc = e % GT;
                Xs[rr][cc] = (r + rr < r1 && ti + cc < c1) ? X[(r + rr) * ldx + ti + cc] : 0.0;
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int k = 0; k < GK; ++k) {
                    double a[4], b[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] = Xs[k][4 * by + i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) b[j] = Xs[k][4 * bx + j];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(a[i], b[j], acc[i][j]);
                }
            }
            __syncthreads();
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int gi = ti + 4 * by + i, gj = tj + 4 * bx + j;
                    if (gi < c1 && gj < c2) partials[((size_t)blockIdx.z * c1 + gi) * c2 + gj] = acc[i][j];
                }
        }
        return;
    }
    for (int64_t r = r0; r < r1; r += GK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q, rr = e / GT, cc = e % GT;
            const bool rowok = r + rr < r1;
            Xs[rr][cc] = (rowok && ti + cc < c1) ? X[(r + rr) * ldx + ti + cc] : 0.0;
            Ys[rr][cc] = (rowok && tj + cc < c2) ? Y[(r + rr) * ldy + tj + cc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Xs[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Ys[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gi = ti + ty + 16 * i, gj = tj + tx + 16 * j;
            if (gi < c1 && gj < c2) partials[((size_t)blockIdx.z * c1 + gi) * c2 + gj] = acc[i][j];
        }
}

// G = sum of the chunk partials in chunk order. sym: only tiles with
// row tile <= column tile were computed; the rest is mirrored.
__global__ void k_sum_partials(const double* __restrict__ partials, int nchunks, int c1, int c2, int sym,
                               double* __restrict__ G) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t count = (int64_t)c1 * c2;
    if (e >= count) return;
    int i = (int)(e / c2), j = (int)(e % c2);
    if (sym && i > j) { const int t = i; i = j; j = t; }   // lower entries mirror the upper ones
    const int64_t src = (int64_t)i * c2 + j;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += partials[(size_t)c * count + src];
    G[e] = s;
}

static void gram_plan(int c1, int c2, int64_t n, int sm_count, int* nchunks, int64_t* rpc, int sym = 0) {
    const int tx = (c1 + GT - 1) / GT;
    const int tiles = sym ? tx * (tx + 1) / 2 : tx * ((c2 + GT - 1) / GT);
    // at most 4 working CTAs per SM (256 threads x 64 registers each fill the register file),
    // rounded DOWN so tiles x chunks fits one wave: a few CTAs of a second wave would cost
    // a whole CTA's time at a quarter of the SM's FP64 issue rate
    int64_t want = 4 * (int64_t)sm_count / tiles;
    int64_t maxc = (n + 63) / 64;
    if (want > maxc) want = maxc;
    if (want < 1) want = 1;
    int64_t r = (n + want - 1) / want;
    r = (r + GK - 1) / GK * GK;
    if (r < GK) r = GK;
    *rpc = r;
    *nchunks = (int)((n + r - 1) / r);
    if (*nchunks < 1) *nchunks = 1;
}

size_t gram_partials_size(int c1, int c2, int64_t n, int sm_count, int sym) {
    int nc;
    int64_t rpc;
    gram_plan(c1, c2, n, sm_count, &nc, &rpc, sym);
    return (size_t)nc * c1 * c2;
}

// Upper bound of gram_partials_size(c', c', n) over every c' <= c: the chunk
// count is at most 4 sm / tiles + 1 and c'^2 / tiles <= 2 * 64^2 (symmetric tiles).
size_t gram_partials_cap(int c, int sm_count) {
    const size_t tiles = (size_t)((c + GT - 1) / GT) * ((c + GT - 1) / GT);
    return (size_t)(4 * sm_count + 1) * GT * GT * 2 + tiles * GT * GT;
}

int gram(const double* X, int64_t ldx, int c1, const double* Y, int64_t ldy, int c2, int64_t n, double* G,
         double* partials, size_t partials_cap, int sm_count, cudaStream_t s) {
    cmsvd_context* ctx = current_ctx();
    if (ctx && ctx->s == s && ozaki_applies(ctx, n, c1, c2)) return gram_ozaki(ctx, X, ldx, c1, Y, ldy, c2, n, G, c2);
    int nc;
    int64_t rpc;
    const int sym = (X == Y && c1 == c2 && ldx == ldy) ? 1 : 0;
    gram_plan(c1, c2, n, sm_count, &nc, &rpc, sym);
    if ((size_t)nc * c1 * c2 > partials_cap) { set_error("gram scratch too small"); return CMSVD_WORKSPACE_TOO_SMALL; }
    dim3 grid((c1 + GT - 1) / GT, (c2 + GT - 1) / GT, nc);
    const int64_t cnt = (int64_t)c1 * c2;
    const double tiles = (double)grid.x * grid.y, tiles_done = sym ? grid.x * (grid.x + 1) / 2.0 : tiles;
    {
        ProfScope ps(CMSVD_PROF_GRAM, s, 8.0 * n * (sym ? c1 : c1 + c2) + 8.0 * cnt,
                     2.0 * n * c1 * c2 * tiles_done / tiles, 2);
        k_gram_partial<<<grid, 256, 0, s>>>(X, ldx, c1, Y, ldy, c2, n, rpc, sym, partials);
        CM_LAUNCH();
        k_sum_partials<<<(int)((cnt + 255) / 256), 256, 0, s>>>(partials, nc, c1, c2, sym, G);
        CM_LAUNCH();
    }
    return CMSVD_OK;
}

// ----------------------------------------------------------------------------- Z = X W
// upper != 0: W is upper triangular, so column tile [cc0, cc0+64) needs k < cc0 + 64 only.
__global__ void __launch_bounds__(256) k_gemm_nn(const double* __restrict__ X, int64_t ldx, const double* __restrict__ W,
                                                 int64_t ldw, double* __restrict__ Z, int64_t ldz, int64_t n, int c1, int c2,
                                                 int upper) {
    __shared__ double Xs[GT][GK + 1];
    __shared__ double Ws[GK][GT];
    const int64_t r0 = (int64_t)blockIdx.y * GT;
    const int cc0 = blockIdx.x * GT;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    const int kend = upper ? min(c1, cc0 + GT) : c1;
    for (int k0 = 0; k0 < kend; k0 += GK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int xr = e / GK, xk = e % GK;
            Xs[xr][xk] = (r0 + xr < n && k0 + xk < c1) ? X[(r0 + xr) * ldx + k0 + xk] : 0.0;
            const int wk = e / GT, wc = e % GT;
            Ws[wk][wc] = (k0 + wk < c1 && cc0 + wc < c2) ? W[(int64_t)(k0 + wk) * ldw + cc0 + wc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Xs[ty + 16 * i][k];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Ws[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gr = r0 + ty + 16 * i;
            const int gc = cc0 + tx + 16 * j;
            if (gr < n && gc < c2) Z[gr * ldz + gc] = acc[i][j];
        }
}

int gemm_nn(const double* X, int64_t ldx, const double* W, int64_t ldw, double* Z, int64_t ldz, int64_t n, int c1,
            int c2, cudaStream_t s, int upper) {
    if (n <= 0 || c2 <= 0) return CMSVD_OK;
    cmsvd_context* ctx = current_ctx();
    if (ctx && ctx->s == s && ozaki_applies(ctx, n, c1, c2)) return gemm_ozaki(ctx, X, ldx, W, ldw, Z, ldz, n, c1, c2);
    dim3 grid((c2 + GT - 1) / GT, (unsigned)((n + GT - 1) / GT));
    double work = 0.0;   // multiply-adds actually performed per row
    for (int cc0 = 0; cc0 < c2; cc0 += GT) work += (double)(upper ? min(c1, cc0 + GT) : c1) * min(GT, c2 - cc0);
    ProfScope ps(CMSVD_PROF_GEMM, s, 8.0 * ((double)n * c1 + (double)c1 * c2 + (double)n * c2), 2.0 * n * work);
    // few output tiles and a long contraction (the c x c products): the library GEMM spreads
    // the contraction over the GPU (dense arithmetic 1 keeps the tiled kernel throughout)
    if (ctx && ctx->s == s && ctx->dense_arith == 0 && !upper && c1 >= 128 && (int64_t)grid.x * grid.y < ctx->sm_count &&
        n < (1ll << 31) && ldx < (1ll << 31) && ldw < (1ll << 31) && ldz < (1ll << 31))
        return gemm_fp64_small(ctx, X, ldx, W, ldw, Z, ldz, n, c1, c2);
    k_gemm_nn<<<grid, 256, 0, s>>>(X, ldx, W, ldw, Z, ldz, n, c1, c2, upper);
    CM_LAUNCH();
    return CMSVD_OK;
}

// ----------------------------------------------------------------------------- Cholesky / inverse
// R (c x c, row-major, upper) with R^T R = G + shift I, where
// shift = shift_coef * trace(G) (shift_coef = 0: plain Cholesky). One CTA.
// A pivot that is not positive is replaced by a tiny positive value and flagged.
__global__ void __launch_bounds__(1024) k_chol(const double* __restrict__ G, int c, double shift_coef, double* __restrict__ R,
                                               int* flag) {
    __shared__ double sh_tr, sh_piv;
    const int t = threadIdx.x, nt = blockDim.x;
    if (t == 0) {
        double tr = 0.0;
        for (int i = 0; i < c; ++i) tr += G[(size_t)i * c + i];
        sh_tr = tr;
    }
    __syncthreads();
    const double shift = shift_coef * sh_tr;
    for (int e = t; e < c * c; e += nt) {
        const int i = e / c, j = e % c;
        R[e] = j >= i ? G[e] + (i == j ? shift : 0.0) : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < c; ++k) {
        if (t == 0) {
            double p = R[(size_t)k * c + k];
            const double floor_ = 1e-300 + 1e-32 * sh_tr;
            if (!(p > floor_)) {
                atomicOr(flag, 1);
                p = floor_;
            }
            const double rp = rsqrt(p);
            R[(size_t)k * c + k] = p * rp;
            sh_piv = rp;
        }
        __syncthreads();
        const double rpiv = sh_piv;
        for (int j = k + 1 + t; j < c; j += nt) R[(size_t)k * c + j] *= rpiv;
        __syncthreads();
        for (int i = k + 1 + (t >> 5); i < c; i += nt >> 5) {
            const double rki = R[(size_t)k * c + i];
            for (int j = i + (t & 31); j < c; j += 32) R[(size_t)i * c + j] = __fma_rn(-rki, R[(size_t)k * c + j], R[(size_t)i * c + j]);
        }
        __syncthreads();
    }
}

// Ri = R^{-1} for upper-triangular R (row-major, c <= 1024): one 128-thread CTA per column j
// solves R x = e_j in the column (axpy) form: for k = j, j-1, .., 0, x_k is final once the
// columns right of it have been subtracted, x_k *= 1/R_kk, and every row i < k takes
// x_i -= R_ik x_k (each thread owns rows t + 128 u). A step is one FP64 multiply, one FMA per
// owned row and one barrier, rather than a block reduction (an FP64 add costs ~64 clocks of
// latency on GB300); the next column of R is loaded during the current step, and the
// reciprocals of the diagonal are formed first, in parallel.
constexpr int TI_RPT = 8;   // rows per thread
__global__ void __launch_bounds__(128) k_trinv(const double* __restrict__ R, int c, double* __restrict__ Ri) {
    __shared__ double x[128 * TI_RPT];
    __shared__ double rinv[128 * TI_RPT];
    const int j = blockIdx.x, t = threadIdx.x;
    if (j >= c) return;
    for (int i = t; i < c; i += 128) Ri[(size_t)i * c + j] = 0.0;
    for (int i = t; i <= j; i += 128) {
        rinv[i] = 1.0 / R[(size_t)i * c + i];
        x[i] = i == j ? 1.0 : 0.0;
    }
    double rc[TI_RPT];   // R[i][k] of the owned rows for the current k
#pragma unroll
    for (int u = 0; u < TI_RPT; ++u) {
        const int i = t + 128 * u;
        rc[u] = i < j ? R[(size_t)i * c + j] : 0.0;
    }
    __syncthreads();
    for (int k = j; k >= 0; --k) {
        const double xk = x[k] * rinv[k];
        double rn[TI_RPT];
#pragma unroll
        for (int u = 0; u < TI_RPT; ++u) {
            const int i = t + 128 * u;
            rn[u] = i < k - 1 ? __ldg(R + (size_t)i * c + (k - 1)) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < TI_RPT; ++u) {
            const int i = t + 128 * u;
            if (i < k) x[i] = __fma_rn(-rc[u], xk, x[i]);
        }
        __syncthreads();   // every thread has read x[k] and updated its rows
        if (t == 0) x[k] = xk;
#pragma unroll
        for (int u = 0; u < TI_RPT; ++u) rc[u] = rn[u];
    }
    __syncthreads();
    for (int i = t; i <= j; i += 128) Ri[(size_t)i * c + j] = x[i];
}

// ----------------------------------------------------------------------------- one-sided Jacobi SVD
constexpr int JC_MAXDIM = 1024;             // L M <= 512; the dense direct solver factors n <= 1024
// The cols columns (length rows) of Bm (rows x cols, row-major) are copied to Xc
// (column-major) and rotated pairwise until mutually orthogonal (Hestenes):
// Bm V = Xc, so sv_j = ||Xc_j|| are the singular values (zero when cols > rows),
// Xc_j / sv_j the left and V_j the right singular vectors. Round-robin
// ordering; one warp per pair; perm sorts sv descending (stable).
__global__ void __launch_bounds__(1024) k_jacobi(double* __restrict__ Xc, int rows, int cols, double* __restrict__ V,
                                                 const double* __restrict__ fro2, double tol, double* __restrict__ sv,
                                                 int* __restrict__ perm) {
    __shared__ int rotated;
    const int t = threadIdx.x, nt = blockDim.x;
    const int lane = t & 31, warp = t >> 5, nwarps = nt >> 5;
    const int np = (cols + 1) / 2 * 2;            // players (one dummy when cols is odd)
    const double negl = 1e-36 * *fro2;
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (t == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < np - 1; ++round) {
            for (int k = warp; k < np / 2; k += nwarps) {
                int p, q;
                if (k == 0) { p = round; q = np - 1; }
                else { p = (round + k) % (np - 1); q = (round - k + (np - 1)) % (np - 1); }
                if (p >= cols || q >= cols) continue;
                if (p > q) { int tmp = p; p = q; q = tmp; }
                double* xp = Xc + (size_t)p * rows;
                double* xq = Xc + (size_t)q * rows;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = lane; i < rows; i += 32) {
                    const double a = xp[i], b = xq[i];
                    al = __fma_rn(a, a, al);
                    be = __fma_rn(b, b, be);
                    ga = __fma_rn(a, b, ga);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                if (fabs(ga) > tol * sqrt(al * be) && al > negl && be > negl) {
                    const double zeta = (be - al) / (2.0 * ga);
                    const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
                    for (int i = lane; i < rows; i += 32) {
                        const double a = xp[i], b = xq[i];
                        xp[i] = cs * a - sn * b;
                        xq[i] = sn * a + cs * b;
                    }
                    double* vp = V + (size_t)p * cols;
                    double* vq = V + (size_t)q * cols;
                    for (int i = lane; i < cols; i += 32) {
                        const double va = vp[i], vb = vq[i];
                        vp[i] = cs * va - sn * vb;
                        vq[i] = sn * va + cs * vb;
                    }
                    if (lane == 0) rotated = 1;
                }
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    for (int j = warp; j < cols; j += nwarps) {
        double s2 = 0.0;
        for (int i = lane; i < rows; i += 32) s2 = __fma_rn(Xc[(size_t)j * rows + i], Xc[(size_t)j * rows + i], s2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) sv[j] = sqrt(s2);
    }
    __syncthreads();
    // perm: descending sv, ties by index (a stable sort), each position found by counting. A
    // nonnegative double orders like its bit pattern, so the comparisons are integer ones (a
    // serial insertion sort with FP64 compares took ~1 ms at 256 columns on GB300).
    __shared__ long long key[JC_MAXDIM];
    for (int i = t; i < cols; i += blockDim.x) key[i] = __double_as_longlong(sv[i]);
    __syncthreads();
    for (int i = t; i < cols; i += blockDim.x) {
        const long long ki = key[i];
        int r = 0;
        for (int j = 0; j < cols; ++j) r += key[j] > ki || (key[j] == ki && j < i);
        perm[r] = i;
    }
}

// Grid barrier for cooperative launches (all CTAs co-resident: cudaLaunchCooperativeKernel
// refuses otherwise). The last CTA to arrive resets the arrival count and advances the
// generation word, which the others poll; polling a word that is written once per barrier,
// rather than the count every CTA increments, keeps the atomics uncontended (a variant that
// polled the count made the 256 x 256 Jacobi 10% slower). The wait has an iteration limit:
// past it the kernel sets ctl[3] (timeout), and every CTA leaves at the next barrier.
// ctl: [0] arrivals, [1] generation, [2] sweeps done (Jacobi), [3] timeout.
__device__ __forceinline__ bool grid_barrier(unsigned* ctl, unsigned nblocks) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = ctl + 1;
        volatile unsigned* err = ctl + 3;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(ctl, 1u) == nblocks - 1) {
            atomicExch(ctl, 0u);
            __threadfence();
            atomicAdd(ctl + 1, 1u);
        } else {
            long long it = 0;
            while (*gen == g && *err == 0) {
                if (++it > 20000000LL) { atomicExch(ctl + 3, 1u); break; }   // >= 0.8 s
                if (it > 2048) __nanosleep(40);   // poll hot first: a round lasts microseconds
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile unsigned*)(ctl + 3) == 0;
}


// Cooperative form for 97..1024 columns: one CTA per pair of a round (round-robin ordering,
// the pairs of a round are disjoint), all sweeps in one launch. A column and its V column
// travel between the CTAs that own them in consecutive rounds through a mailbox in L2 that
// carries its own synchronization: every FP64 value is stored as two 8-byte words, each
// holding 32 bits of the value and the 32-bit version of the column (the rounds that have
// updated it). Naturally aligned 8-byte accesses are single-copy atomic, so a reader that
// sees the expected version in both words of an element has that element's new value; the
// owner of a pair in round r polls its two columns until every word carries version r,
// rotates them, and stores them back with version r + 1 (the same layout as the low-latency
// protocol of NCCL). A round then needs no memory fence and no separate flag: one
// store-to-load trip through L2. Each column is read and written once per round, by the
// owner of its pair, who is also its next writer, so one mailbox slot per column is
// enough. One bounded grid barrier per sweep decides convergence (did any CTA rotate).
// Columns whose squared norm is below negl (1e-36 ||Bm||_F^2) are treated as zero.
// GB300 runs an FP64 warp instruction in 16 clocks whatever its active lanes, and a
// dependent FP64 operation takes ~64 clocks (rsqrt ~440, sqrt and division ~650-700;
// measured), so the three dot products are summed over the block with 6 FP64 additions a
// warp, and only warp 0 computes the rotation (two reciprocal square roots, see below),
// shared through shared memory. Per round that chain, not the wait for the partner
// columns, is most of the time (measured on a 256 x 256 problem: 4.5 us a round with the
// plain shuffle sums and a division-and-square-root angle, 4.4 us of it without the waits,
// 1.3 us without the sums and the angle; 3.6 us as written). Exact 128-bit integer dot
// products in block fixed point, tried in place of the FP64 sums, were 12% slower.
// (Measured alternatives,
// slower on this part: an 8-CTA thread-block cluster keeping column blocks in shared
// memory, 25-36 ms per 256 x 256 SVD, FP64-bound on its 8 SMs; block-cyclic cooperative
// kernels with 2 or 4 columns per block, 31 and 21 ms; this form with a grid barrier per
// round, 16 ms; with per-column version counters and fences, 15 ms.)
// Every wait is bounded: past the limit a CTA sets ctl[3] and every CTA leaves.
// RPT: rows (and V entries) per thread, the smallest of 2, 4, 8 with 128 RPT >= rows, cols.
// Mailbox column j: 128 RPT X elements, then 128 RPT V elements, 16 bytes each, at
// mb + j 256 RPT.
__host__ __device__ constexpr int jc_rpt(int mx) { return mx <= 256 ? 2 : mx <= 512 ? 4 : 8; }

size_t jacobi_scratch_words(int dim) {
    // 64 control words (ctl, one rotation word per sweep), then the mailbox (byte 256 on)
    return 64 + (size_t)dim * 256 * jc_rpt(dim) * 4;
}

__device__ __forceinline__ ulonglong2 mb_ld(const ulonglong2* a) {
    ulonglong2 r;
    asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(r.x), "=l"(r.y) : "l"(a) : "memory");
    return r;
}
__device__ __forceinline__ void mb_st(ulonglong2* a, double v, unsigned ver) {
    const unsigned long long f = (unsigned long long)ver << 32;
    const unsigned long long hi = f | (unsigned)__double2hiint(v), lo = f | (unsigned)__double2loint(v);
    asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(a), "l"(hi), "l"(lo) : "memory");
}
__device__ __forceinline__ bool mb_is(ulonglong2 w, unsigned ver) {
    return (unsigned)(w.x >> 32) == ver && (unsigned)(w.y >> 32) == ver;
}
__device__ __forceinline__ double mb_val(ulonglong2 w) { return __hiloint2double((int)(unsigned)w.x, (int)(unsigned)w.y); }

// Polls this thread's elements of columns p (into a) and q (into b, when two) until all carry
// version ver. Elements: slot u < RPT is X row threadIdx.x + 128 u, slot RPT + u the V entry.
// For RPT = 8 the elements are polled in four batches (the registers in flight: 512 columns
// need 4 co-resident CTAs per SM, 128 registers a thread).
// Returns nonzero on timeout or when another CTA has set ctl[3].
template <int RPT>
__device__ __forceinline__ int mb_wait(const ulonglong2* cp, const ulonglong2* cq, bool two, int rows, int cols,
                                       unsigned ver, const unsigned* ctl, double (&a)[2 * RPT], double (&b)[2 * RPT]) {
    constexpr int SLOTS = 2 * RPT, BATCH = RPT >= 8 ? 4 : 2 * RPT;
#pragma unroll
    for (int s0 = 0; s0 < SLOTS; s0 += BATCH) {
        long long it = 0;
        for (;;) {
            ulonglong2 wa[BATCH], wb[BATCH];
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const int sl = s0 + k, u = sl < RPT ? sl : sl - RPT;
                const int i = threadIdx.x + 128 * u, lim = sl < RPT ? rows : cols;
                const int off = (sl < RPT ? 0 : 128 * RPT) + i;
                if (i < lim) {
                    wa[k] = mb_ld(cp + off);
                    if (two) wb[k] = mb_ld(cq + off);
                }
            }
            bool ok = true;
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const int sl = s0 + k, u = sl < RPT ? sl : sl - RPT;
                const int i = threadIdx.x + 128 * u, lim = sl < RPT ? rows : cols;
                a[sl] = 0.0;
                b[sl] = 0.0;
                if (i < lim) {
                    ok = ok && mb_is(wa[k], ver);
                    a[sl] = mb_val(wa[k]);
                    if (two) {
                        ok = ok && mb_is(wb[k], ver);
                        b[sl] = mb_val(wb[k]);
                    }
                }
            }
            if (ok) break;
            if (++it > 2000000LL) return 1;   // about a second of L2 polls
            if ((it & 1023) == 0 && *(volatile const unsigned*)(ctl + 3) != 0) return 1;
        }
    }
    return 0;
}

// Sums three values over a 128-thread block with 6 FP64 additions a warp instead of 15: the
// first two shuffle levels exchange halves of the value set, so lanes 0-7 go on with a, 8-15
// with b, 16-23 with c; warp 0 then adds the four warps' totals. Fixed order: deterministic.
// The sums are valid in warp 0 only.
__device__ __forceinline__ void block_sum3_128_w0(double& a, double& b, double& c, double (*sh)[4]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool h4 = lane & 16, h3 = lane & 8;
    double k0 = h4 ? c : a, k1 = h4 ? 0.0 : b;
    const double s0 = h4 ? a : c, s1 = h4 ? b : 0.0;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    double v = h3 ? k1 : k0;
    v += __shfl_xor_sync(0xffffffffu, h3 ? k0 : k1, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    if ((lane & 7) == 0 && lane < 24) sh[lane >> 3][w] = v;
    __syncthreads();
    if (w == 0) {
        const int vi = lane < 3 ? lane : 0;
        const double t = (sh[vi][0] + sh[vi][1]) + (sh[vi][2] + sh[vi][3]);
        a = __shfl_sync(0xffffffffu, t, 0);
        b = __shfl_sync(0xffffffffu, t, 1);
        c = __shfl_sync(0xffffffffu, t, 2);
    }
}

template <int RPT>
__global__ void __launch_bounds__(128, RPT >= 8 ? 4 : 1) k_jacobi_coop(ulonglong2* __restrict__ mb, double* __restrict__ Xc,
                                                     double* __restrict__ V, int rows, int cols, int np, double tol,
                                                     const double* __restrict__ fro2, int max_sweeps, unsigned* ctl,
                                                     unsigned* rot) {
    constexpr int CS = 256 * RPT;   // mailbox column stride (elements)
    __shared__ double sh[3][4];
    __shared__ double sh_cs, sh_sn;
    __shared__ int sh_ok;
    // the X columns are scaled by sc = 2^-e (exact) when first loaded, so that the scaled
    // ||Bm||_F lies in [1/2, 1), and scaled back by 2^e when unpacked
    const double f2 = *fro2;
    int e2 = 0;
    if (f2 > 0.0 && f2 <= 1.7e308) frexp(sqrt(f2), &e2);
    const double sc = ldexp(1.0, -e2);
    const double negl = 1e-36 * (f2 * sc * sc);
    const double tol2 = tol * tol;
    const int k = blockIdx.x;
    int sweep = 0;
    bool rotated = false;   // this CTA rotated in the current sweep (thread 0)
    for (; sweep < max_sweeps; ++sweep) {
        for (int round = 0; round < np - 1; ++round) {
            const unsigned ver = (unsigned)(sweep * (np - 1) + round);
            int p, q;
            if (k == 0) { p = round; q = np - 1; }
            else { p = (round + k) % (np - 1); q = (round - k + (np - 1)) % (np - 1); }
            if (p > q) { const int t = p; p = q; q = t; }
            // p < cols always; q = cols is the padding column (odd cols), which has no data
            const bool two = q < cols;
            ulonglong2* cp = mb + (size_t)p * CS;
            ulonglong2* cq = mb + (size_t)(two ? q : p) * CS;
            double xa[2 * RPT], xb[2 * RPT];   // [0, RPT): X rows, [RPT, 2 RPT): V entries
            const int fail = mb_wait<RPT>(cp, cq, two, rows, cols, ver, ctl, xa, xb);
            if (ver == 0) {   // every column is in exactly one pair of the first round
#pragma unroll
                for (int u = 0; u < RPT; ++u) {
                    xa[u] *= sc;
                    xb[u] *= sc;
                }
            }
            if (__syncthreads_or(fail)) {
                if (threadIdx.x == 0) atomicExch(ctl + 3, 1u);
                return;
            }
            double cs = 1.0, sn = 0.0;
            if (two) {
                double dal = 0.0, dbe = 0.0, dga = 0.0;
#pragma unroll
                for (int u = 0; u < RPT; ++u) {
                    dal = __fma_rn(xa[u], xa[u], dal);
                    dbe = __fma_rn(xb[u], xb[u], dbe);
                    dga = __fma_rn(xa[u], xb[u], dga);
                }
                block_sum3_128_w0(dal, dbe, dga, sh);
                if (threadIdx.x < 32) {
                    // |ga| > tol sqrt(al be), without the square root (the columns are scaled so
                    // that ||Bm||_F is in [1/2, 1): no overflow here)
                    const int ok = dga * dga > tol2 * (dal * dbe) && dal > negl && dbe > negl;
                    // The rotation that zeroes ga: cot(2 theta) = zeta = (be - al) / (2 ga), |theta| <= pi/4,
                    // tan(theta) = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)). With h = sqrt(d^2 + 4 ga^2),
                    // d = be - al: cos(2 theta) = |d| / h, sin(2 theta) = sign(zeta) 2 |ga| / h, and the
                    // half-angle forms cos(theta) = sqrt((1 + cos 2 theta) / 2), sin(theta) =
                    // sin(2 theta) / (2 cos theta) need two reciprocal square roots and no division,
                    // a shorter chain of dependent FP64 operations than tan(theta) and 1 / sqrt(1 + t^2).
                    // Computed unconditionally and selected by ok.
                    const double d = dbe - dal, g2 = 2.0 * dga;
                    const double sgn = (d == 0.0 || (d > 0.0) == (dga > 0.0)) ? 1.0 : -1.0;
                    const double ri = rsqrt(__fma_rn(d, d, g2 * g2));
                    const double c2 = fabs(d) * ri, s2 = sgn * fabs(g2) * ri;
                    const double hc = __fma_rn(c2, 0.5, 0.5), w = rsqrt(hc);
                    const double c = ok ? hc * w : 1.0, sg = ok ? 0.5 * s2 * w : 0.0;
                    if (threadIdx.x == 0) {
                        sh_ok = ok;
                        sh_cs = c;
                        sh_sn = sg;
                        rotated = rotated || ok;
                    }
                }
                __syncthreads();
                if (sh_ok) {
                    cs = sh_cs;
                    sn = sh_sn;
                }
            }
            // publish version ver + 1 (unchanged values when no rotation)
#pragma unroll
            for (int sl = 0; sl < 2 * RPT; ++sl) {
                const int u = sl < RPT ? sl : sl - RPT;
                const int i = threadIdx.x + 128 * u, lim = sl < RPT ? rows : cols;
                if (i < lim) {
                    const int off = (sl < RPT ? 0 : 128 * RPT) + i;
                    if (two) {
                        mb_st(cp + off, cs * xa[sl] - sn * xb[sl], ver + 1);
                        mb_st(cq + off, sn * xa[sl] + cs * xb[sl], ver + 1);
                    } else {
                        mb_st(cp + off, xa[sl], ver + 1);
                    }
                }
            }
        }
        if (threadIdx.x == 0 && rotated) atomicExch(rot + sweep, 1u);
        rotated = false;
        if (!grid_barrier(ctl, gridDim.x)) return;   // every rotation of the sweep is counted
        if (*(volatile unsigned*)(rot + sweep) == 0) { ++sweep; break; }
    }
    // the barrier above ordered every final store before these loads
    const double usc = ldexp(1.0, e2);
    for (int j = k; j < cols; j += gridDim.x) {
        const ulonglong2* c = mb + (size_t)j * CS;
        for (int i = threadIdx.x; i < rows; i += 128) Xc[(size_t)j * rows + i] = usc * mb_val(mb_ld(c + i));
        for (int i = threadIdx.x; i < cols; i += 128) V[(size_t)j * cols + i] = mb_val(mb_ld(c + 128 * RPT + i));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl[2] = sweep;
}

__global__ void __launch_bounds__(1024) k_jacobi_finish(const double* __restrict__ Xc, int rows, int cols,
                                                        double* __restrict__ sv, int* __restrict__ perm) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x >> 5;
    for (int j = warp; j < cols; j += nwarps) {
        double s2 = 0.0;
        for (int i = lane; i < rows; i += 32) s2 = __fma_rn(Xc[(size_t)j * rows + i], Xc[(size_t)j * rows + i], s2);
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) sv[j] = sqrt(s2);
    }
    __syncthreads();
    // perm: descending sv, ties by index (a stable sort), each position found by counting. A
    // nonnegative double orders like its bit pattern, so the comparisons are integer ones (a
    // serial insertion sort with FP64 compares took ~1 ms at 256 columns on GB300).
    __shared__ long long key[JC_MAXDIM];
    for (int i = t; i < cols; i += blockDim.x) key[i] = __double_as_longlong(sv[i]);
    __syncthreads();
    for (int i = t; i < cols; i += blockDim.x) {
        const long long ki = key[i];
        int r = 0;
        for (int j = 0; j < cols; ++j) r += key[j] > ki || (key[j] == ki && j < i);
        perm[r] = i;
    }
}

// Rotates the columns of Bm (trans = 0; Bm V = Xc) or of Bm^T (trans = 1; Bm^T V = Xc,
// so Bm = V diag(sv) (Xc / sv)^T: V holds the LEFT singular vectors of Bm). Applying
// the method to the transpose of the R factors met here roughly halves the sweeps.
// With a mailbox (mb != nullptr, the cooperative form) Xc and V are written there, version 0.
__global__ void k_jacobi_init_t(const double* __restrict__ Bm, int brows, int bcols, int trans, double* __restrict__ Xc,
                                double* __restrict__ V, double* __restrict__ fro2, ulonglong2* __restrict__ mb, int rpt) {
    const int rows = trans ? bcols : brows, cols = trans ? brows : bcols;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t e = t0; e < (int64_t)brows * bcols; e += nt) {
        const int i = (int)(e / bcols), j = (int)(e % bcols);     // Bm(i, j)
        const int c = trans ? i : j, r = trans ? j : i;          // column c, row r of the rotated matrix
        if (mb) mb_st(mb + (size_t)c * 256 * rpt + r, Bm[e], 0u);
        else Xc[(size_t)c * rows + r] = Bm[e];
    }
    for (int64_t e = t0; e < (int64_t)cols * cols; e += nt) {
        const double v = (e / cols == e % cols) ? 1.0 : 0.0;
        if (mb) mb_st(mb + (size_t)(e / cols) * 256 * rpt + 128 * rpt + e % cols, v, 0u);
        else V[e] = v;
    }
    if (blockIdx.x == 0) {
        __shared__ double sh[32];
        double acc = 0.0;
        for (int64_t e = threadIdx.x; e < (int64_t)brows * bcols; e += blockDim.x) acc = __fma_rn(Bm[e], Bm[e], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
            *fro2 = t;
        }
    }
}

int jacobi_svd(const double* Bm, int brows, int bcols, int trans, double* Xc, double* V, double* sv, int* perm,
               int* flag2, cmsvd_context* ctx, double tol_in, unsigned* jac_ctl) {
    cudaStream_t s = ctx->s;
    const int rows = trans ? bcols : brows, cols = trans ? brows : bcols;
    double* fro2 = (double*)(flag2 + 2);   // flag2: 16 bytes of scratch (int rotated, pad, double)
    if (rows > JC_MAXDIM || cols > JC_MAXDIM) { set_error("Jacobi SVD supports at most %d rows and columns", JC_MAXDIM); return CMSVD_NOT_SUPPORTED; }
    // jac_ctl: 64 control words, then the mailbox of the cooperative form (16-byte aligned)
    ulonglong2* mb = cols > 96 ? reinterpret_cast<ulonglong2*>(jac_ctl + 64) : nullptr;
    {
        ProfScope ps(CMSVD_PROF_JACOBI, s, 16.0 * rows * cols + 8.0 * cols * cols, 0.0);
        k_jacobi_init_t<<<64, 256, 0, s>>>(Bm, brows, bcols, trans, Xc, V, fro2, mb, jc_rpt(rows > cols ? rows : cols));
        CM_LAUNCH();
    }
    const int np = (cols + 1) / 2 * 2;
    const double tol = tol_in > 0.0 ? tol_in : fmax(1e-15, rows * 2.220446049250313e-16);
    if (cols <= 96) {
        ProfScope ps(CMSVD_PROF_JACOBI, s, 16.0 * (rows + cols) * cols, 0.0);
        k_jacobi<<<1, 1024, 0, s>>>(Xc, rows, cols, V, fro2, tol, sv, perm);
        CM_LAUNCH();
        return CMSVD_OK;
    }
    // all sweeps in one launch; ctl (4 words) and rot (one word per sweep) lead jac_ctl
    unsigned* ctl = jac_ctl;
    unsigned* rot = jac_ctl + 4;
    const int max_sweeps = 40;
    CM_CUDA(cudaMemsetAsync(ctl, 0, sizeof(unsigned) * 64, s));
    const int grid = np / 2;
    {
        const int mx = rows > cols ? rows : cols;
        const void* fn = mx <= 256 ? (const void*)k_jacobi_coop<2>
                       : mx <= 512 ? (const void*)k_jacobi_coop<4> : (const void*)k_jacobi_coop<8>;
        int per_sm = 0;
        CM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 128, 0));
        if (per_sm * ctx->sm_count < grid) { set_error("Jacobi grid of %d CTAs cannot be co-resident", grid); return CMSVD_NOT_SUPPORTED; }
        ProfScope ps(CMSVD_PROF_JACOBI, s, 0.0, 0.0, 1);
        void* args[] = {&mb, &Xc, &V, (void*)&rows, (void*)&cols, (void*)&np, (void*)&tol, &fro2, (void*)&max_sweeps, &ctl,
                        &rot};
        CM_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(128), args, 0, s));
        note_launch();
    }
    unsigned h[4];
    CM_CUDA(cudaMemcpyAsync(ctx->pinned, ctl, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, s));
    CM_CUDA(cudaStreamSynchronize(s));
    memcpy(h, ctx->pinned, sizeof(h));
    if (h[3]) { set_error("Jacobi SVD: a wait between rounds timed out"); return CMSVD_CUDA_ERROR; }
    // account the work of the sweeps that ran
    {
        Profiler& pr = prof();
        if (pr.timing && pr.nrec > 0 && pr.recs[pr.nrec - 1].cls == CMSVD_PROF_JACOBI) {
            const double pairs = (double)h[2] * (np - 1.0) * (np / 2);
            pr.recs[pr.nrec - 1].bytes = pairs * 16.0 * (rows + cols);
            pr.recs[pr.nrec - 1].flops = pairs * (6.0 * rows + 6.0 * (rows + cols));
        }
    }
    ProfScope ps(CMSVD_PROF_JACOBI, s, 8.0 * rows * cols, 2.0 * rows * cols);
    k_jacobi_finish<<<1, 1024, 0, s>>>(Xc, rows, cols, sv, perm);
    CM_LAUNCH();
    return CMSVD_OK;
}

// ----------------------------------------------------------------------------- orthogonalization

// min over max of the diagonal of an upper-triangular R (condition estimate of CholeskyQR)
// Cooperative blocked form of k_chol for larger c (same result up to rounding order):
// panels of CB = 32 rows. Per panel: CTA 0 factors the diagonal block in shared memory;
// every thread of the grid solves one column of the panel row R12 = R11^{-T} A12 in
// registers, against the diagonal block staged in each CTA's shared memory (column form:
// one dependent multiply-add per step instead of a dot-product chain per row); the grid
// updates the upper triangle of the trailing block, A22 -= R12^T R12. GB300 issues only 2
// FP64 FMA per clock per SM and a dependent FP64 operation takes ~64 clocks, so the c^3/6
// multiply-adds are spread over the whole grid and the serial steps kept out of L2. The
// grid barrier between phases is bounded (ctl[3] = 1 on timeout; every CTA then returns).
constexpr int CB = 32;
__global__ void __launch_bounds__(256) k_chol_coop(const double* __restrict__ G, int c, double shift_coef,
                                                   double* __restrict__ R, int* flag, unsigned* ctl) {
    __shared__ double sh_tr, sh_rpiv;
    __shared__ double Ds[CB][CB + 1];   // the panel's diagonal block (upper triangle)
    __shared__ double rdiag[CB];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + t, gthreads = (int64_t)gridDim.x * blockDim.x;
    if (wid == 0) {   // trace of G: lanes over the diagonal, then a fixed shuffle tree
        double tr = 0.0;
        for (int i = lane; i < c; i += 32) tr += G[(size_t)i * c + i];
        for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
        if (lane == 0) sh_tr = tr;
    }
    __syncthreads();
    const double shift = shift_coef * sh_tr;
    const double floor_ = 1e-300 + 1e-32 * sh_tr;
    for (int e = (int)gtid; e < c * c; e += (int)gthreads) {
        const int i = e / c, j = e % c;
        R[e] = j >= i ? G[e] + (i == j ? shift : 0.0) : 0.0;
    }
    if (!grid_barrier(ctl, gridDim.x)) return;
    // R is written by other CTAs between the barriers: it is read with __ldcg (from L2)
    for (int k0 = 0; k0 < c; k0 += CB) {
        const int b = min(CB, c - k0), w = c - k0 - b;
        if (blockIdx.x == 0) {   // diagonal block, right-looking, in shared memory
            for (int e = t; e < b * b; e += blockDim.x) {
                const int i = e / b, j = e % b;
                Ds[i][j] = j >= i ? __ldcg(R + (size_t)(k0 + i) * c + k0 + j) : 0.0;
            }
            __syncthreads();
            for (int kk = 0; kk < b; ++kk) {
                if (t == 0) {
                    double p = Ds[kk][kk];
                    if (!(p > floor_)) {
                        atomicOr(flag, 1);
                        p = floor_;
                    }
                    const double rp = rsqrt(p);
                    Ds[kk][kk] = p * rp;
                    sh_rpiv = rp;
                }
                __syncthreads();
                const double rpiv = sh_rpiv;
                for (int j = kk + 1 + t; j < b; j += blockDim.x) Ds[kk][j] *= rpiv;
                __syncthreads();
                for (int i = kk + 1 + wid; i < b; i += nw) {
                    const double rki = Ds[kk][i];
                    for (int j = i + lane; j < b; j += 32) Ds[i][j] = __fma_rn(-rki, Ds[kk][j], Ds[i][j]);
                }
                __syncthreads();
            }
            for (int e = t; e < b * b; e += blockDim.x) {
                const int i = e / b, j = e % b;
                if (j >= i) R[(size_t)(k0 + i) * c + k0 + j] = Ds[i][j];
            }
        }
        if (!grid_barrier(ctl, gridDim.x)) return;
        if (w == 0) break;
        // panel row: column j of R12 solves R11^T x = A12(:, j) by forward substitution in
        // registers, in column (axpy) form: x_i = a_i / R_ii, then a_q -= R_iq x_i for q > i
        // (the same multiply-adds, in the same order, as the row form)
        for (int e = t; e < b * b; e += blockDim.x) {
            const int i = e / b, j = e % b;
            Ds[i][j] = j >= i ? __ldcg(R + (size_t)(k0 + i) * c + k0 + j) : 0.0;
        }
        __syncthreads();
        for (int i = t; i < b; i += blockDim.x) rdiag[i] = 1.0 / Ds[i][i];
        __syncthreads();
        for (int64_t jj = gtid; jj < w; jj += gthreads) {
            const int j = k0 + b + (int)jj;
            double av[CB];
#pragma unroll
            for (int u = 0; u < CB; ++u) av[u] = u < b ? __ldcg(R + (size_t)(k0 + u) * c + j) : 0.0;
#pragma unroll
            for (int i = 0; i < CB; ++i) {
                if (i < b) {
                    const double x = av[i] * rdiag[i];
                    av[i] = x;
#pragma unroll
                    for (int q = i + 1; q < CB; ++q) av[q] = __fma_rn(-Ds[i][q], x, av[q]);
                }
            }
#pragma unroll
            for (int u = 0; u < CB; ++u)
                if (u < b) R[(size_t)(k0 + u) * c + j] = av[u];
        }
        if (!grid_barrier(ctl, gridDim.x)) return;
        // trailing update of the upper triangle: a warp per row, lanes over its columns
        for (int64_t gw = gtid >> 5; gw < w; gw += gthreads >> 5) {
            const int i = k0 + b + (int)gw;
            for (int j = i + lane; j < c; j += 32) {
                double acc = __ldcg(R + (size_t)i * c + j);
                for (int q = k0; q < k0 + b; ++q)
                    acc = __fma_rn(-__ldcg(R + (size_t)q * c + i), __ldcg(R + (size_t)q * c + j), acc);
                R[(size_t)i * c + j] = acc;
            }
        }
        if (!grid_barrier(ctl, gridDim.x)) return;
    }
}

// Deflation by Cholesky with diagonal pivoting of G = T^T T (c <= 512, one CTA): at step k
// the largest remaining diagonal entry is brought to position k; the factorization stops
// when it is <= keep * max diag(G). Then P^T G P ~ L L^T with L (c x c') and a discarded
// Schur complement of trace <= (c - c') keep max diag(G). Only the upper triangle of the
// working copy W is kept (the symmetric swap reads the mirrored entries). Outputs:
// R3 = L^T P^T (c' x c, row-major; T ~ (T T3) R3), Lt = L11^T (c' x c', row-major, in W),
// perm (the pivot order, c ints, in the L scratch) and c'. T3 = P_1 L11^{-T} is formed by
// k_pchol_t3 from the inverse of Lt, so that (T T3)^T (T T3) = I.
// Ties pick the smaller index, so the result is deterministic.
__global__ void __launch_bounds__(1024) k_pchol_deflate(const double* __restrict__ G, int c, double keep,
                                                        double* __restrict__ W, double* __restrict__ L,
                                                        double* __restrict__ R3, int* __restrict__ cp_out) {
    __shared__ int perm[512];
    __shared__ double lcol[512];
    __shared__ long long rv[32];
    __shared__ int ri[32];
    __shared__ double sh_d0, sh_piv, sh_lkk, sh_rl;
    __shared__ int sh_j;
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5, nw = nt >> 5;
    for (int e = t; e < c * c; e += nt) {
        W[e] = G[e];
        L[e] = 0.0;
    }
    for (int i = t; i < c; i += nt) perm[i] = i;
    __syncthreads();
    int k = 0;
    for (; k <= c; ++k) {
        // argmax of the remaining diagonal (k == 0 also gives max diag(G))
        // (on the bit patterns: a positive double orders like its bits, a negative one below
        // every positive; FP64 compares cost 16 clocks a warp instruction on GB300)
        long long best = LLONG_MIN;
        int bi = c;
        for (int i = k + t; i < c; i += nt) {
            const long long d = __double_as_longlong(W[(size_t)i * c + i]);
            if (d > best) { best = d; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
        __syncthreads();
        if (t == 0) {
            long long bv = rv[0];
            int bj = ri[0];
            for (int w = 1; w < nw; ++w)
                if (rv[w] > bv || (rv[w] == bv && ri[w] < bj)) { bv = rv[w]; bj = ri[w]; }
            const double dv = bj < c ? __longlong_as_double(bv) : -1.0;
            if (k == 0) sh_d0 = dv;
            sh_piv = dv;
            sh_j = bj;
            const double rl = rsqrt(dv);   // one reciprocal square root: 1/l and l = d / l
            sh_lkk = dv * rl;
            sh_rl = rl;
        }
        __syncthreads();
        const int j = sh_j;
        const double d = sh_piv;
        if (k == c || !(d > keep * sh_d0)) break;
        if (j != k) {   // symmetric swap of indices k < j on the upper triangle
            for (int x = k + 1 + t; x < c; x += nt) {
                if (x == j) continue;
                double* a = W + (size_t)k * c + x;
                double* b = x < j ? W + (size_t)x * c + j : W + (size_t)j * c + x;
                const double tmp = *a;
                *a = *b;
                *b = tmp;
            }
            for (int col = t; col < k; col += nt) {
                const double a = L[(size_t)k * c + col];
                L[(size_t)k * c + col] = L[(size_t)j * c + col];
                L[(size_t)j * c + col] = a;
            }
            if (t == 0) {
                const double a = W[(size_t)k * c + k];
                W[(size_t)k * c + k] = W[(size_t)j * c + j];
                W[(size_t)j * c + j] = a;
                const int pa = perm[k];
                perm[k] = perm[j];
                perm[j] = pa;
            }
            __syncthreads();
        }
        const double lkk = sh_lkk, rl = sh_rl;
        for (int i = k + t; i < c; i += nt) {
            const double v = i == k ? lkk : W[(size_t)k * c + i] * rl;
            L[(size_t)i * c + k] = v;
            lcol[i] = v;   // column k of L, staged for the update (its global copy is strided)
        }
        __syncthreads();
        // trailing upper triangle: a warp per row, lanes over its columns (no index division,
        // no idle lanes below the diagonal)
        for (int i = k + 1 + warp; i < c; i += nw) {
            const double lik = lcol[i];
            for (int jj = i + lane; jj < c; jj += 32)
                W[(size_t)i * c + jj] = __fma_rn(-lik, lcol[jj], W[(size_t)i * c + jj]);
        }
        __syncthreads();
    }
    const int cp = k;
    if (t == 0) *cp_out = cp;
    for (int e = t; e < cp * c; e += nt) {       // R3 row-major cp x c: R3[i][perm[r]] = L[r][i]
        const int i = e / c, r = e % c;
        R3[(size_t)i * c + perm[r]] = r >= i ? L[(size_t)r * c + i] : 0.0;
    }
    for (int e = t; e < cp * cp; e += nt) {      // Lt = L11^T, row-major cp x cp, into W
        const int i = e / cp, jj = e % cp;
        W[e] = jj >= i ? L[(size_t)jj * c + i] : 0.0;
    }
    __syncthreads();
    int* perm_out = (int*)L;
    for (int i = t; i < c; i += nt) perm_out[i] = perm[i];
}

// T3 (c x cp, row-major) = P_1 L11^{-T}: row perm[r] is row r of Lti = (L11^T)^{-1} for r < cp,
// the other rows are zero.
__global__ void k_pchol_t3(const double* __restrict__ Lti, int cp, const int* __restrict__ perm, int c,
                           double* __restrict__ T3) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c * cp; e += gridDim.x * blockDim.x) {
        const int r = e / cp, i = e % cp;
        T3[(size_t)perm[r] * cp + i] = r < cp ? Lti[(size_t)r * cp + i] : 0.0;
    }
}

__global__ void k_diag_ratio(const double* __restrict__ R, int c, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo = 1e300, hi = 0.0;
    for (int i = 0; i < c; ++i) {
        const double d = fabs(R[(size_t)i * c + i]);
        lo = fmin(lo, d);
        hi = fmax(hi, d);
    }
    *out = hi > 0.0 ? lo / hi : 0.0;
}

size_t orth_scratch(int c, int64_t n, int sm_count) {
    return (size_t)n * c + 14 * (size_t)c * c + 2 * (size_t)c + gram_partials_cap(c, sm_count) + 256;
}

namespace {
struct OrthCtx {
    cmsvd_context* ctx;
    cudaStream_t s;
    double *G, *Ri, *part;
    size_t pcap;
    int* flag;       // device int
    int64_t n;
    unsigned* ctl;   // 4 device words for the cooperative Cholesky
};

// Launches k_chol (c <= 64) or k_chol_coop; ctl: 4 device words of scratch.
int chol_launch(cmsvd_context* ctx, cudaStream_t s, const double* G, int c, double coef, double* R, int* flag,
                unsigned* ctl) {
    CM_CUDA(cudaMemsetAsync(ctl, 0, 4 * sizeof(unsigned), s));
    ProfScope ps(CMSVD_PROF_SMALL, s, 16.0 * c * c, c * (double)c * c / 3.0);
    if (c <= 64) {
        k_chol<<<1, 1024, 0, s>>>(G, c, coef, R, flag);
        CM_LAUNCH();
        return CMSVD_OK;
    }
    int per_sm = 0;   // queried per call: cheap, and safe when several host threads solve at once
    CM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_coop, 256, 0));
    int grid = ctx->sm_count < 128 ? ctx->sm_count : 128;
    if (per_sm * ctx->sm_count < grid) grid = per_sm * ctx->sm_count;
    if (grid < 1) { set_error("Cholesky grid cannot be co-resident"); return CMSVD_NOT_SUPPORTED; }
    void* args[] = {(void*)&G, (void*)&c, (void*)&coef, (void*)&R, (void*)&flag, (void*)&ctl};
    CM_CUDA(cudaLaunchCooperativeKernel((const void*)k_chol_coop, dim3(grid), dim3(256), args, 0, s));
    note_launch();
    return CMSVD_OK;
}

// R (cc x cc) with R^T R = G + shift I. base = 0: plain Cholesky first. A failed
// attempt (non-positive pivot) is repeated with a 100x larger shift, starting from
// 10 (cc + sqrt(n)) u trace(G) -- the size of the rounding error of a computed Gram.
int chol_adaptive(OrthCtx& o, int cc, bool shifted, double* R) {
    const double u = 1.1102230246251565e-16;
    double coef = shifted ? 10.0 * (cc + sqrt((double)o.n)) * u : 0.0;
    for (int attempt = 0; attempt < 12; ++attempt) {
        CM_CUDA(cudaMemsetAsync(o.flag, 0, sizeof(int), o.s));
        CM_TRY(chol_launch(o.ctx, o.s, o.G, cc, coef, R, o.flag, o.ctl));
        CM_CUDA(cudaMemcpyAsync(o.ctx->pinned, o.flag, 4 * sizeof(int), cudaMemcpyDeviceToHost, o.s));
        CM_CUDA(cudaMemcpyAsync(o.ctx->pinned + 4, o.ctl, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, o.s));
        CM_CUDA(cudaStreamSynchronize(o.s));
        if (o.ctx->pinned[4 + 3]) { set_error("Cholesky grid barrier timed out"); return CMSVD_CUDA_ERROR; }
        if (o.ctx->pinned[0] == 0) return CMSVD_OK;
        coef = coef > 0.0 ? coef * 100.0 : 10.0 * (cc + sqrt((double)o.n)) * u;
    }
    set_error("Cholesky of a Gram matrix failed for every shift");
    return CMSVD_BREAKDOWN;
}

int trinv(OrthCtx& o, const double* R, int cc) {
    ProfScope ps(CMSVD_PROF_SMALL, o.s, 16.0 * cc * cc, cc * (double)cc * cc / 3.0);
    k_trinv<<<cc, 128, 0, o.s>>>(R, cc, o.Ri);
    CM_LAUNCH();
    return CMSVD_OK;
}

// one CholeskyQR pass: Xout = Xin R^{-1}, R^T R = Xin^T Xin (+ shift)
int cholqr_pass(OrthCtx& o, const double* Xin, int64_t ldi, int cc, bool shifted, double* R, double* Xout) {
    CM_TRY(gram(Xin, ldi, cc, Xin, ldi, cc, o.n, o.G, o.part, o.pcap, o.ctx->sm_count, o.s));
    CM_TRY(chol_adaptive(o, cc, shifted, R));
    CM_TRY(trinv(o, R, cc));
    CM_TRY(gemm_nn(Xin, ldi, o.Ri, cc, Xout, cc, o.n, cc, cc, o.s, 1));
    return CMSVD_OK;
}
}  // namespace

// X (n x c, ldx) = Q R with Q (n x c', ld c') orthonormal and R (c' x c, row-major).
//   deflate = 0: when the first plain Cholesky succeeds and diag(R) spans less than
//   1e5 (cond(X) well below 1/sqrt(u)), CholeskyQR2 is used (c' = c).
//   Otherwise: two shifted CholeskyQR passes bring every direction of X whose
//   singular value exceeds ~1e-14 ||X|| to O(1); a pivoted Cholesky of the Gram of the
//   result deflates the directions left at rounding level; a congruence polish (from
//   that same Gram) and one plain pass from the data restore orthogonality to working
//   precision.
int orth_qr(const double* X, int64_t ldx, int64_t n, int c, double* Q, double* R, int* c_out, double* scratch, int* ints,
            int deflate, cmsvd_context* ctx, double* Rcorr, bool r_from_gram) {
    cudaStream_t s = ctx->s;
    double* T = scratch;
    double* G = T + (size_t)n * c;
    double* R1 = G + (size_t)c * c;
    double* R2 = R1 + (size_t)c * c;
    double* R3 = R2 + (size_t)c * c;
    double* R4 = R3 + (size_t)c * c;
    double* R5 = R4 + (size_t)c * c;
    double* Ri = R5 + (size_t)c * c;
    double* Wp = Ri + (size_t)c * c;     // pivoted-Cholesky scratch (c x c each)
    double* Lp = Wp + (size_t)c * c;
    double* T3 = Lp + (size_t)c * c;
    double* M1 = T3 + (size_t)c * c;
    double* M2 = M1 + (size_t)c * c;
    double* part = M2 + (size_t)c * c;
    OrthCtx o{ctx, s, G, Ri, part, gram_partials_cap(c, ctx->sm_count), ints, n, (unsigned*)(ints + 4)};
    int* cp_dev = ints + 1;
    double* ratio = (double*)(ints + 2);
    if (!deflate) {
        // CholeskyQR2 attempt
        CM_TRY(gram(X, ldx, c, X, ldx, c, n, G, part, o.pcap, ctx->sm_count, s));
        CM_CUDA(cudaMemsetAsync(o.flag, 0, sizeof(int), s));
        CM_TRY(chol_launch(ctx, s, G, c, 0.0, R1, o.flag, o.ctl));
        {
            ProfScope ps(CMSVD_PROF_SMALL, s, 8.0 * c, 0.0);
            k_diag_ratio<<<1, 32, 0, s>>>(R1, c, ratio);
            CM_LAUNCH();
        }
        CM_CUDA(cudaMemcpyAsync(ctx->pinned, ints, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CM_CUDA(cudaStreamSynchronize(s));
        if (ctx->pinned[4 + 3]) { set_error("Cholesky grid barrier timed out"); return CMSVD_CUDA_ERROR; }
        double rat;
        memcpy(&rat, ctx->pinned + 2, sizeof(double));
        if (ctx->pinned[0] == 0 && r_from_gram && !Rcorr) {
            // the caller bounded the Gram's rounding error below its accuracy target: R = R1
            CM_CUDA(cudaMemcpyAsync(R, R1, sizeof(double) * (size_t)c * c, cudaMemcpyDeviceToDevice, s));
            *c_out = c;
            return CMSVD_OK;
        }
        if (ctx->pinned[0] == 0 && rat > 1e-5) {
            // Q1 = X R1^{-1}; its Gram gives R2; Q = Q1 R2^{-1} is left implicit
            double* Q1 = Rcorr ? Q : T;
            CM_TRY(trinv(o, R1, c));
            CM_TRY(gemm_nn(X, ldx, Ri, c, Q1, c, n, c, c, s, 1));
            CM_TRY(gram(Q1, c, c, Q1, c, c, n, G, part, o.pcap, ctx->sm_count, s));
            CM_TRY(chol_adaptive(o, c, false, R2));
            if (Rcorr) {
                CM_TRY(trinv(o, R2, c));
                CM_CUDA(cudaMemcpyAsync(Rcorr, Ri, sizeof(double) * (size_t)c * c, cudaMemcpyDeviceToDevice, s));
            }
            CM_TRY(gemm_nn(R2, c, R1, c, R, c, c, c, c, s));
            *c_out = c;
            return CMSVD_OK;
        }
    }
    // two shifted passes: X -> Q (R1), Q -> T (R2)
    CM_TRY(cholqr_pass(o, X, ldx, c, true, R1, Q));
    CM_TRY(cholqr_pass(o, Q, c, c, true, R2, T));
    // deflation: the directions of T left at rounding level (Gram pivots <= 1e-10 of the
    // largest) are separated from the O(1) ones by a pivoted Cholesky of its Gram
    CM_TRY(gram(T, c, c, T, c, c, n, G, part, o.pcap, ctx->sm_count, s));
    if (c > 512) { set_error("orthogonalization supports at most 512 columns"); return CMSVD_NOT_SUPPORTED; }
    {
        ProfScope ps(CMSVD_PROF_SMALL, s, 40.0 * c * c, c * (double)c * c / 6.0);
        k_pchol_deflate<<<1, 1024, 0, s>>>(G, c, 1e-10, Wp, Lp, R3, cp_dev);
        CM_LAUNCH();
    }
    CM_CUDA(cudaMemcpyAsync(ctx->pinned, cp_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CM_CUDA(cudaStreamSynchronize(s));
    const int cp = ctx->pinned[0];
    *c_out = cp;
    if (cp <= 0) return CMSVD_OK;
    CM_TRY(trinv(o, Wp, cp));   // (L11^T)^{-1} into o.Ri
    {
        ProfScope ps(CMSVD_PROF_SMALL, s, 16.0 * c * cp, 0.0);
        k_pchol_t3<<<(c * cp + 255) / 256, 256, 0, s>>>(o.Ri, cp, (const int*)Lp, c, T3);
        CM_LAUNCH();
    }
    // first plain pass without forming Q3 = T T3: its Gram is T3^T (T^T T) T3, from the Gram
    // of T computed above (error amplified by at most 1 / lambda_min of the kept directions,
    // <= 1e10 u, which only affects Q4's orthogonality), so Q4 = T (T3 R4^{-1}) is one GEMM
    CM_TRY(gemm_nn(G, c, T3, cp, M1, cp, c, c, cp, s));                 // G T3 (c x cp)
    CM_TRY(gram(T3, cp, cp, M1, cp, cp, c, M2, part, o.pcap, ctx->sm_count, s));   // T3^T G T3 (cp x cp)
    {
        // chol_adaptive factors o.G; point it at the small Gram
        double* g_saved = o.G;
        o.G = M2;
        const int st = chol_adaptive(o, cp, false, R4);
        o.G = g_saved;
        CM_TRY(st);
    }
    CM_TRY(trinv(o, R4, cp));
    CM_TRY(gemm_nn(T3, cp, Ri, cp, M1, cp, c, cp, cp, s, 1));          // T3 R4^{-1} (c x cp)
    CM_TRY(gemm_nn(T, c, M1, cp, Q, cp, n, c, cp, s));                 // Q4 = T (T3 R4^{-1})
    // plain pass from data: Gram(Q4) = R5^T R5; Q = Q4 R5^{-1} is left implicit
    CM_TRY(gram(Q, cp, cp, Q, cp, cp, n, G, part, o.pcap, ctx->sm_count, s));
    CM_TRY(chol_adaptive(o, cp, false, R5));
    if (Rcorr) {
        CM_TRY(trinv(o, R5, cp));
        CM_CUDA(cudaMemcpyAsync(Rcorr, Ri, sizeof(double) * (size_t)cp * cp, cudaMemcpyDeviceToDevice, s));
    }
    // R = R5 R4 R3 R2 R1
    CM_TRY(gemm_nn(R2, c, R1, c, M1, c, c, c, c, s));
    CM_TRY(gemm_nn(R3, c, M1, c, M2, c, cp, c, c, s));
    CM_TRY(gemm_nn(R4, cp, M2, c, M1, c, cp, cp, c, s));
    CM_TRY(gemm_nn(R5, cp, M1, c, R, c, cp, cp, c, s));
    return CMSVD_OK;
}

}  // namespace cmsvd

// ============================================================================= allocation-free Gram
// Scratch for the chunk partials of cmsvd_gram_noalloc: a fixed device array in
// this file (8 MiB, present on every GPU that loads the library, until exit).
namespace cmsvd {
namespace {
constexpr int64_t kNoAllocDoubles = int64_t(1) << 20;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};   // per device: device address of the array
}  // namespace
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// The host-side name of a __device__ array is not a device address. Resolve the
// address once per device, with that device current.
static int noalloc_scratch(int device, double** out) {
    if (device < 0 || device >= 256) { set_error("device ordinal %d out of range", device); return CMSVD_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        g_noalloc_ptr[device] = (double*)p;
    }
    *out = g_noalloc_ptr[device];
    return CMSVD_OK;
}

}  // namespace cmsvd

extern "C" int cmsvd_gram_noalloc(cmsvd_context* ctx, int64_t n, int32_t c1, int32_t c2, const double* X, int64_t ldx,
                                  const double* Y, int64_t ldy, double* G) {
    using namespace cmsvd;
    if (!ctx || !X || !Y || !G) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    if (n < 1 || c1 < 1 || c2 < 1 || c1 > 4096 || c2 > 4096 || ldx < c1 || ldy < c2) {
        set_error("need n >= 1, 1 <= c1, c2 <= 4096, ldx >= c1, ldy >= c2");
        return CMSVD_INVALID_ARG;
    }
    if ((int64_t)c1 * c2 > kNoAllocDoubles) {
        set_error("c1*c2 = %lld exceeds the %lld-entry static scratch of cmsvd_gram_noalloc; use cmsvd_gram",
                  (long long)c1 * c2, (long long)kNoAllocDoubles);
        return CMSVD_INVALID_ARG;
    }
    Session se;
    CM_TRY(se.open(ctx));   // the context's device is current from here to the return
    double* scratch = nullptr;
    CM_TRY(noalloc_scratch(ctx->device, &scratch));
    const int sym = (X == Y && c1 == c2 && ldx == ldy) ? 1 : 0;
    int nc;
    int64_t rpc;
    gram_plan(c1, c2, n, ctx->sm_count, &nc, &rpc, sym);
    const int64_t maxc = kNoAllocDoubles / ((int64_t)c1 * c2);   // chunks that fit the array
    if (nc > maxc) {
        rpc = (n + maxc - 1) / maxc;
        rpc = (rpc + GK - 1) / GK * GK;
        nc = (int)((n + rpc - 1) / rpc);
    }
    dim3 grid((c1 + GT - 1) / GT, (c2 + GT - 1) / GT, nc);
    const int64_t cnt = (int64_t)c1 * c2;
    // every partial that k_sum_partials reads is written first: nothing needs clearing
    k_gram_partial<<<grid, 256, 0, ctx->s>>>(X, ldx, c1, Y, ldy, c2, n, rpc, sym, scratch);
    CM_LAUNCH();
    k_sum_partials<<<(int)((cnt + 255) / 256), 256, 0, ctx->s>>>(scratch, nc, c1, c2, sym, G);
    CM_LAUNCH();
    return se.close();
}
