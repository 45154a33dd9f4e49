// Direct shifted solves for matrices whose column graph splits into small
// connected components (Alg. 1 / Alg. 2 steps 1-2 with exact solves, as in the
// paper's experiments, which solve every system directly).
//
// Columns that share a row are connected; A^T A is block diagonal over the
// components, so (s_j I - A^T A)^{-1} X splits into independent small solves.
// Each component's H_c = A_c^T A_c (s x s) is factored once, independently of
// the shift, as H_c = W diag(lambda) W^T (cyclic Jacobi in one warp). Then
//   (s_j I - H_c)^{-1} = W diag(1 / (s_j - lambda)) W^T
// for every shift, and with the halving of Sec. 3.1 and the iteration
// technique (Eqs. iter1-iter2) the moment block of the component is
//   S_k = W diag( c_k(lambda) f(lambda)^(ell-1) ) W^T X_c,
//   c_k(lambda) = 2 Re sum_j w_j m_j^k / (s_j - lambda),  f = c_0.
// The analysis (finding the components) runs once per matrix on the host,
// like the symbolic phase of a sparse direct solver; the numeric work runs on
// the device. The dense direct solver (n <= 1024, one large component) is at the
// end of this file.
#include "internal.cuh"
#include <vector>
#include <numeric>
#include <algorithm>

namespace cmsvd {

void components_free(Components* c) {
    if (c->cols) cudaFree(c->cols);
    if (c->comp_row_ptr) cudaFree(c->comp_row_ptr);
    if (c->comp_rows) cudaFree(c->comp_rows);
    if (c->comp_first_dev) cudaFree(c->comp_first_dev);
    if (c->col_local) cudaFree(c->col_local);
    free(c->group_size);
    free(c->group_count);
    free(c->group_col_off);
    free(c->comp_first);
    *c = Components();
}

static int64_t uf_find(std::vector<int64_t>& p, int64_t x) {
    while (p[x] != x) {
        p[x] = p[p[x]];
        x = p[x];
    }
    return x;
}

int components_build(cmsvd_matrix* M) {
    cmsvd_context* ctx = M->ctx;
    const int64_t m = M->A.m, n = M->A.n, nnz = M->A.nnz;
    std::vector<int64_t> rowptr(m + 1);
    std::vector<int32_t> colidx(nnz > 0 ? nnz : 1);
    CM_CUDA(cudaMemcpyAsync(rowptr.data(), M->A.rowptr, sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToHost, ctx->s));
    if (nnz > 0) CM_CUDA(cudaMemcpyAsync(colidx.data(), M->A.colidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, ctx->s));
    CM_CUDA(cudaStreamSynchronize(ctx->s));
    std::vector<int64_t> par(n);
    std::iota(par.begin(), par.end(), 0);
    for (int64_t i = 0; i < m; ++i) {
        if (rowptr[i + 1] <= rowptr[i]) continue;
        int64_t r0 = uf_find(par, colidx[rowptr[i]]);
        for (int64_t p = rowptr[i] + 1; p < rowptr[i + 1]; ++p) {
            int64_t r1 = uf_find(par, colidx[p]);
            if (r1 != r0) {
                if (r1 < r0) std::swap(r0, r1);
                par[r1] = r0;
            }
        }
    }
    // component ids in order of their smallest column
    std::vector<int64_t> cid(n, -1), root_id(n, -1);
    int64_t count = 0;
    for (int64_t c = 0; c < n; ++c) {
        int64_t r = uf_find(par, c);
        if (root_id[r] < 0) root_id[r] = count++;
        cid[c] = root_id[r];
    }
    std::vector<int64_t> size(count, 0);
    for (int64_t c = 0; c < n; ++c) size[cid[c]]++;
    // order components by (size, id)
    std::vector<int64_t> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return size[x] < size[y]; });
    std::vector<int64_t> pos(count);
    for (int64_t k = 0; k < count; ++k) pos[order[k]] = k;
    std::vector<int64_t> first(count + 1, 0);
    for (int64_t k = 0; k < count; ++k) first[k + 1] = first[k] + size[order[k]];
    std::vector<int32_t> cols(n), local(n);
    std::vector<int64_t> fill(count, 0);
    for (int64_t c = 0; c < n; ++c) {
        const int64_t k = pos[cid[c]];
        local[c] = (int32_t)fill[k];
        cols[first[k] + fill[k]++] = (int32_t)c;
    }
    // rows bucketed by component (rows in ascending order within a component)
    std::vector<int64_t> rptr(count + 1, 0);
    for (int64_t i = 0; i < m; ++i)
        if (rowptr[i + 1] > rowptr[i]) rptr[pos[cid[colidx[rowptr[i]]]] + 1]++;
    for (int64_t k = 0; k < count; ++k) rptr[k + 1] += rptr[k];
    std::vector<int32_t> rows(rptr[count] > 0 ? rptr[count] : 1);
    std::vector<int64_t> rfill(rptr.begin(), rptr.end() - 1);
    for (int64_t i = 0; i < m; ++i)
        if (rowptr[i + 1] > rowptr[i]) rows[rfill[pos[cid[colidx[rowptr[i]]]]]++] = (int32_t)i;
    // groups of equal size
    std::vector<int32_t> gsize;
    std::vector<int64_t> gcount, goff;
    for (int64_t k = 0; k < count;) {
        int64_t s = size[order[k]], e = k;
        while (e < count && size[order[e]] == s) ++e;
        gsize.push_back((int32_t)s);
        gcount.push_back(e - k);
        goff.push_back(k);   // first component index of the group
        k = e;
    }
    Components& C = M->comp;
    components_free(&C);
    C.count = count;
    C.max_size = count ? size[order[count - 1]] : 0;
    C.n_groups = (int64_t)gsize.size();
    C.group_size = (int32_t*)malloc(sizeof(int32_t) * (gsize.size() + 1));
    C.group_count = (int64_t*)malloc(sizeof(int64_t) * (gsize.size() + 1));
    C.group_col_off = (int64_t*)malloc(sizeof(int64_t) * (gsize.size() + 1));
    C.comp_first = (int64_t*)malloc(sizeof(int64_t) * (count + 1));
    if (!C.group_size || !C.group_count || !C.group_col_off || !C.comp_first) { set_error("host allocation failed"); return CMSVD_OUT_OF_MEMORY; }
    for (size_t g = 0; g < gsize.size(); ++g) {
        C.group_size[g] = gsize[g];
        C.group_count[g] = gcount[g];
        C.group_col_off[g] = goff[g];
    }
    memcpy(C.comp_first, first.data(), sizeof(int64_t) * (count + 1));
    CM_CUDA(cudaMalloc(&C.cols, sizeof(int32_t) * n));
    CM_CUDA(cudaMalloc(&C.col_local, sizeof(int32_t) * n));
    CM_CUDA(cudaMalloc(&C.comp_row_ptr, sizeof(int64_t) * (count + 1)));
    CM_CUDA(cudaMalloc(&C.comp_rows, sizeof(int32_t) * rows.size()));
    CM_CUDA(cudaMalloc(&C.comp_first_dev, sizeof(int64_t) * (count + 1)));
    CM_CUDA(cudaMemcpyAsync(C.cols, cols.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->s));
    CM_CUDA(cudaMemcpyAsync(C.col_local, local.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->s));
    CM_CUDA(cudaMemcpyAsync(C.comp_row_ptr, rptr.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, ctx->s));
    CM_CUDA(cudaMemcpyAsync(C.comp_rows, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, ctx->s));
    CM_CUDA(cudaMemcpyAsync(C.comp_first_dev, first.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, ctx->s));
    CM_CUDA(cudaStreamSynchronize(ctx->s));
    C.ready = true;
    return CMSVD_OK;
}

size_t direct_workspace(const cmsvd_matrix*, const cmsvd_params*) { return 4096; }

// ----------------------------------------------------------------------------- kernel
// One warp per component of size s (<= 32). Shared memory per warp:
// H (s x s), W (s x s), rowvec (s), coef (Mk x s), P (s x L).
struct DirectArgs {
    const int64_t* rowptr;
    const int32_t* colidx;
    const double* vals;
    const int32_t* cols;
    const int32_t* col_local;
    const int64_t* comp_row_ptr;
    const int32_t* comp_rows;
    const int64_t* comp_first;
    const double2* quad;
    const double* X;
    int64_t ldx;
    double* S;
    int64_t lds;
    int64_t comp0;     // first component of the group
    int64_t ncomp;
    int s, L, J, Mk, ell;
};

// c_m(lambda) f(lambda)^(ell-1) for m = 0..Mk-1, with c_m(lambda) = 2 Re sum_j w_j m_j^m / (s_j - lambda)
// and f = c_0 (the filter of Eq. iter1); out[m * stride].
__device__ void filter_coefs(double lam, const double2* __restrict__ quad, int J, int Mk, int ell, double* out,
                             int stride) {
    double f = 0.0;
    for (int m = 0; m < Mk; ++m) out[m * stride] = 0.0;
    for (int j = 0; j < J; ++j) {
        const double2 sh = quad[3 * j], w = quad[3 * j + 1], sc = quad[3 * j + 2];
        // g = w / (s_j - lambda)
        const double dr = sh.x - lam, di = sh.y;
        double gr, gi;
        if (fabs(dr) >= fabs(di)) {
            const double r = di / dr, den = dr + di * r;
            gr = (w.x + w.y * r) / den;
            gi = (w.y - w.x * r) / den;
        } else {
            const double r = dr / di, den = dr * r + di;
            gr = (w.x * r + w.y) / den;
            gi = (w.y * r - w.x) / den;
        }
        f += 2.0 * gr;
        for (int m = 0; m < Mk; ++m) {
            out[m * stride] += 2.0 * gr;
            const double nr = gr * sc.x - gi * sc.y, ni = gr * sc.y + gi * sc.x;
            gr = nr;
            gi = ni;
        }
    }
    double fp = 1.0;
    for (int e = 1; e < ell; ++e) fp *= f;
    for (int m = 0; m < Mk; ++m) out[m * stride] *= fp;
}

__global__ void __launch_bounds__(32) k_direct(DirectArgs a) {
    extern __shared__ double sm[];
    const int s = a.s, L = a.L, lane = threadIdx.x;
    const int64_t q = a.comp0 + blockIdx.x;
    double* H = sm;
    double* W = H + s * s;
    double* rv = W + s * s;
    double* coef = rv + s;
    double* P = coef + a.Mk * s;
    const int32_t* cols = a.cols + a.comp_first[q];
    // H_c = sum over the component's rows of row^T row (rows in ascending order)
    for (int e = lane; e < s * s; e += 32) {
        H[e] = 0.0;
        W[e] = (e / s == e % s) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int64_t rp = a.comp_row_ptr[q]; rp < a.comp_row_ptr[q + 1]; ++rp) {
        const int64_t r = a.comp_rows[rp];
        for (int e = lane; e < s; e += 32) rv[e] = 0.0;
        __syncwarp();
        for (int64_t p = a.rowptr[r] + lane; p < a.rowptr[r + 1]; p += 32) rv[a.col_local[a.colidx[p]]] = a.vals[p];
        __syncwarp();
        for (int e = lane; e < s * s; e += 32) H[e] = __fma_rn(rv[e / s], rv[e % s], H[e]);
        __syncwarp();
    }
    // cyclic Jacobi: H = W diag(lambda) W^T
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int e = lane; e < s * s; e += 32) {
            const int i = e / s, j = e % s;
            if (i < j) off += H[e] * H[e];
            if (i == j) dg += H[e] * H[e];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dg += __shfl_xor_sync(0xffffffffu, dg, o);
        }
        if (off <= 1e-34 * dg || off == 0.0) break;
        for (int p = 0; p < s - 1; ++p) {
            for (int qq = p + 1; qq < s; ++qq) {
                const double apq = H[p * s + qq];
                const double app = H[p * s + p], aqq = H[qq * s + qq];
                if (fabs(apq) <= 1e-300 || fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq))) continue;
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                __syncwarp();
                for (int k = lane; k < s; k += 32) {
                    if (k != p && k != qq) {
                        const double hkp = H[k * s + p], hkq = H[k * s + qq];
                        const double np_ = c * hkp - sn * hkq, nq_ = sn * hkp + c * hkq;
                        H[k * s + p] = np_;
                        H[p * s + k] = np_;
                        H[k * s + qq] = nq_;
                        H[qq * s + k] = nq_;
                    }
                    const double wkp = W[k * s + p], wkq = W[k * s + qq];
                    W[k * s + p] = c * wkp - sn * wkq;
                    W[k * s + qq] = sn * wkp + c * wkq;
                }
                __syncwarp();
                if (lane == 0) {
                    H[p * s + p] = app - t * apq;
                    H[qq * s + qq] = aqq + t * apq;
                    H[p * s + qq] = 0.0;
                    H[qq * s + p] = 0.0;
                }
                __syncwarp();
            }
        }
    }
    __syncwarp();
    // filter-moment coefficients per eigenvalue
    for (int i = lane; i < s; i += 32) filter_coefs(H[i * s + i], a.quad, a.J, a.Mk, a.ell, coef + i, s);
    __syncwarp();
    // P = W^T X_c (s x L), then S rows = W diag(coef_m) P
    for (int l = lane; l < L; l += 32) {
        for (int i = 0; i < s; ++i) {
            double acc = 0.0;
            for (int k = 0; k < s; ++k) acc = __fma_rn(W[k * s + i], a.X[(int64_t)cols[k] * a.ldx + l], acc);
            P[i * L + l] = acc;
        }
    }
    __syncwarp();
    for (int l = lane; l < L; l += 32) {
        for (int k = 0; k < s; ++k) {
            double* srow = a.S + (int64_t)cols[k] * a.lds + l;
            for (int m = 0; m < a.Mk; ++m) {
                double acc = 0.0;
                for (int i = 0; i < s; ++i) acc = __fma_rn(W[k * s + i] * coef[m * s + i], P[i * L + l], acc);
                srow[(int64_t)m * L] = acc;
            }
        }
    }
}

// Components of at most DS_MAX columns: 32 components per warp. The per-component scalar work
// (H_c, its cyclic Jacobi eigendecomposition and the filter-moment coefficients) runs one
// component per lane, so that every FP64 warp instruction does 32 lanes of work (GB300 issues
// FP64 at 2 lanes per clock per SM whatever the active lanes; one warp per component left 28
// of 32 lanes idle on 4-column components). Then the warp goes through its components with
// lanes over the L columns of X for P = W^T X_c and the S rows, as k_direct does. The same
// operations in the same order per component as k_direct. Shared memory, interleaved by
// lane (entry e of lane t at [e 32 + t]): H, W (s x s) and coef (Mk x s) per lane.
constexpr int DS_MAX = 8;
__global__ void __launch_bounds__(32) k_direct_small(DirectArgs a) {
    extern __shared__ double sm[];
    const int s = a.s, L = a.L, lane = threadIdx.x, Mk = a.Mk;
    double* sH = sm;
    double* sW = sH + s * s * 32;
    double* sC = sW + s * s * 32;
    const int64_t q0 = a.comp0 + (int64_t)blockIdx.x * 32;
    const int64_t qend = a.comp0 + a.ncomp;
    const int64_t q = q0 + lane;
#define DS_H(i, j) sH[((i) * s + (j)) * 32 + lane]
#define DS_W(i, j) sW[((i) * s + (j)) * 32 + lane]
    if (q < qend) {
        for (int e = 0; e < s * s; ++e) {
            sH[e * 32 + lane] = 0.0;
            sW[e * 32 + lane] = (e / s == e % s) ? 1.0 : 0.0;
        }
        // H_c = sum over the component's rows of row^T row (rows in ascending order)
        for (int64_t rp = a.comp_row_ptr[q]; rp < a.comp_row_ptr[q + 1]; ++rp) {
            const int64_t r = a.comp_rows[rp];
            const int64_t b = a.rowptr[r], e = a.rowptr[r + 1];
            for (int64_t p1 = b; p1 < e; ++p1) {
                const int i = a.col_local[a.colidx[p1]];
                const double v1 = a.vals[p1];
                for (int64_t p2 = b; p2 < e; ++p2) {
                    const int j = a.col_local[a.colidx[p2]];
                    DS_H(i, j) = __fma_rn(v1, a.vals[p2], DS_H(i, j));
                }
            }
        }
        // cyclic Jacobi: H = W diag(lambda) W^T
        for (int sweep = 0; sweep < 40; ++sweep) {
            double off = 0.0, dg = 0.0;
            for (int i = 0; i < s; ++i)
                for (int j = 0; j < s; ++j) {
                    const double h = DS_H(i, j);
                    if (i < j) off += h * h;
                    if (i == j) dg += h * h;
                }
            if (off <= 1e-34 * dg || off == 0.0) break;
            for (int p = 0; p < s - 1; ++p) {
                for (int qq = p + 1; qq < s; ++qq) {
                    const double apq = DS_H(p, qq);
                    const double app = DS_H(p, p), aqq = DS_H(qq, qq);
                    if (fabs(apq) <= 1e-300 || fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq))) continue;
                    const double theta = (aqq - app) / (2.0 * apq);
                    const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                    for (int k = 0; k < s; ++k) {
                        if (k != p && k != qq) {
                            const double hkp = DS_H(k, p), hkq = DS_H(k, qq);
                            const double np_ = c * hkp - sn * hkq, nq_ = sn * hkp + c * hkq;
                            DS_H(k, p) = np_;
                            DS_H(p, k) = np_;
                            DS_H(k, qq) = nq_;
                            DS_H(qq, k) = nq_;
                        }
                        const double wkp = DS_W(k, p), wkq = DS_W(k, qq);
                        DS_W(k, p) = c * wkp - sn * wkq;
                        DS_W(k, qq) = sn * wkp + c * wkq;
                    }
                    DS_H(p, p) = app - t * apq;
                    DS_H(qq, qq) = aqq + t * apq;
                    DS_H(p, qq) = 0.0;
                    DS_H(qq, p) = 0.0;
                }
            }
        }
        // filter-moment coefficients per eigenvalue: coef(m, i) at sC[(m s + i) 32 + lane]
        for (int i = 0; i < s; ++i) filter_coefs(DS_H(i, i), a.quad, a.J, Mk, a.ell, sC + i * 32 + lane, s * 32);
    }
#undef DS_H
#undef DS_W
    __syncwarp();
    // P = W^T X_c (s values per column l), then S rows = W diag(coef_m) P, component by component
    const int nq = (int)(qend - q0 < 32 ? qend - q0 : 32);
    for (int cq = 0; cq < nq; ++cq) {
        const int32_t* cols = a.cols + a.comp_first[q0 + cq];
        for (int l = lane; l < L; l += 32) {
            double pv[DS_MAX];
#pragma unroll
            for (int i = 0; i < DS_MAX; ++i) {
                double acc = 0.0;
                if (i < s)
                    for (int k = 0; k < s; ++k) acc = __fma_rn(sW[(k * s + i) * 32 + cq], a.X[(int64_t)cols[k] * a.ldx + l], acc);
                pv[i] = acc;
            }
            for (int k = 0; k < s; ++k) {
                double* srow = a.S + (int64_t)cols[k] * a.lds + l;
                for (int m = 0; m < Mk; ++m) {
                    double acc = 0.0;
#pragma unroll
                    for (int i = 0; i < DS_MAX; ++i)
                        if (i < s) acc = __fma_rn(sW[(k * s + i) * 32 + cq] * sC[(m * s + i) * 32 + cq], pv[i], acc);
                    srow[(int64_t)m * L] = acc;
                }
            }
        }
    }
}

int direct_moments(cmsvd_matrix* M, const cmsvd_params* p, const double2* quad, int Mk, const double* X, int64_t ldx,
                   double* S, int64_t lds, Arena& ws) {
    if (!M->comp.ready) CM_TRY(components_build(M));
    const Components& C = M->comp;
    if (C.max_size > 32) {
        set_error("DIRECT solver needs every component of A^T A to have at most 32 columns (largest: %lld)",
                  (long long)C.max_size);
        return CMSVD_NOT_SUPPORTED;
    }
    (void)ws;
    DirectArgs a;
    a.rowptr = M->A.rowptr;
    a.colidx = M->A.colidx;
    a.vals = M->A.vals;
    a.cols = C.cols;
    a.col_local = C.col_local;
    a.comp_row_ptr = C.comp_row_ptr;
    a.comp_rows = C.comp_rows;
    a.comp_first = C.comp_first_dev;
    a.quad = quad;
    a.X = X;
    a.ldx = ldx;
    a.S = S;
    a.lds = lds;
    a.L = p->L;
    a.J = p->N / 2;
    a.Mk = Mk;
    a.ell = p->ell;
    // compulsory traffic: A once, X once, S written once; FP64 flops of the
    // per-component work (H_c, Jacobi sweeps estimated at 6, coefficients, P and S)
    double flops = 0.0;
    for (int64_t g = 0; g < C.n_groups; ++g) {
        const double sz = C.group_size[g], cnt = (double)C.group_count[g];
        flops += cnt * (2.0 * sz * sz * (M->A.m / (double)C.count) + 6.0 * 0.5 * sz * (sz - 1) * 12.0 * sz +
                        sz * a.J * (12.0 + 8.0 * Mk) + 2.0 * sz * sz * a.L * (1.0 + Mk));
    }
    ProfScope ps(CMSVD_PROF_DIRECT, M->ctx->s,
                 12.0 * M->A.nnz + 8.0 * (M->A.m + 1) + 8.0 * M->A.n * a.L + 8.0 * M->A.n * a.L * Mk, flops,
                 C.n_groups);
    for (int64_t g = 0; g < C.n_groups; ++g) {
        a.s = C.group_size[g];
        a.comp0 = C.group_col_off[g];
        a.ncomp = C.group_count[g];
        const size_t smem_small = sizeof(double) * 32 * (2 * a.s * a.s + (size_t)Mk * a.s);
        if (a.s <= DS_MAX && a.ncomp >= 64 && smem_small <= 160 * 1024) {   // 32 components a warp
            const size_t smem = smem_small;
            if (smem > 48 * 1024)
                CM_CUDA(cudaFuncSetAttribute(k_direct_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            const int64_t blocks = (a.ncomp + 31) / 32;
            int64_t done = 0;
            while (done < blocks) {
                const int64_t chunk = blocks - done < 2147483647 ? blocks - done : 2147483647;
                DirectArgs b = a;
                b.comp0 = a.comp0 + done * 32;
                b.ncomp = a.ncomp - done * 32;
                k_direct_small<<<(unsigned)chunk, 32, smem, M->ctx->s>>>(b);
                CM_LAUNCH();
                done += chunk;
            }
            continue;
        }
        const size_t smem = sizeof(double) * (2 * a.s * a.s + a.s + (size_t)Mk * a.s + (size_t)a.s * a.L);
        if (smem > 48 * 1024) CM_CUDA(cudaFuncSetAttribute(k_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int64_t left = a.ncomp;
        int64_t base = a.comp0;
        while (left > 0) {
            const int64_t chunk = left < 2147483647 ? left : 2147483647;
            a.comp0 = base;
            k_direct<<<(unsigned)chunk, 32, smem, M->ctx->s>>>(a);
            CM_LAUNCH();
            base += chunk;
            left -= chunk;
        }
    }
    return CMSVD_OK;
}

// ----------------------------------------------------------------------------- dense direct
// For matrices with few columns (n <= 1024) whose A^T A does not split into small
// components: H = A^T A is formed densely (column blocks of A expanded to dense, then one
// SpMM with A^T each), factored once as H = W diag(lambda) W^T by the one-sided Jacobi
// method (H is symmetric positive semidefinite, so its singular values and right singular
// vectors are its eigenvalues and eigenvectors), and the moments follow as for the
// components above: S_k = W diag(c_k(lambda) f(lambda)^(ell-1)) W^T X.
constexpr int DD_BLOCK = 128;

__global__ void k_expand_cols(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                              const double* __restrict__ vals, int64_t m, int j0, int b, double* __restrict__ D) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const int c = colidx[p] - j0;
            if (c >= 0 && c < b) D[i * b + c] = vals[p];
        }
}

__global__ void k_dense_coef(const double* __restrict__ lam, int n, const double2* __restrict__ quad, int J, int Mk,
                             int ell, double* __restrict__ coef) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        filter_coefs(lam[i], quad, J, Mk, ell, coef + i, n);
}

// Wall[i][m L + l] = coef[m][i] Z[i][l]
__global__ void k_dense_scale(const double* __restrict__ Z, const double* __restrict__ coef, int n, int L, int Mk,
                              double* __restrict__ Wall) {
    const int64_t total = (int64_t)n * L * Mk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ((int64_t)L * Mk)), r = (int)(e % ((int64_t)L * Mk)), mm = r / L, l = r % L;
        Wall[e] = coef[(size_t)mm * n + i] * Z[(size_t)i * L + l];
    }
}

struct DenseBufs { double *D, *H, *Xc, *V, *sv, *coef, *Z, *Wall, *part; int *perm, *ints; unsigned* jctl; size_t pcap; };

static void dense_alloc(DenseBufs& b, Arena& ws, int64_t m, int n, int L, int Mk, int sm) {
    b.D = ws.take<double>((size_t)m * DD_BLOCK);
    b.H = ws.take<double>((size_t)n * n);
    b.Xc = ws.take<double>((size_t)n * n);
    b.V = ws.take<double>((size_t)n * n);
    b.sv = ws.take<double>(n);
    b.coef = ws.take<double>((size_t)n * Mk);
    b.Z = ws.take<double>((size_t)n * L);
    b.Wall = ws.take<double>((size_t)n * L * Mk);
    b.pcap = gram_partials_size(n, L * Mk, n, sm, 0);
    b.part = ws.take<double>(b.pcap);
    b.perm = ws.take<int>(n);
    b.ints = ws.take<int>(16);
    b.jctl = ws.take<unsigned>(jacobi_scratch_words(n));   // Jacobi control words and mailbox
}

size_t dense_workspace(const cmsvd_matrix* M, const cmsvd_params* p) {
    if (M->A.n > 1024) return 0;
    Arena a;
    DenseBufs b;
    dense_alloc(b, a, M->A.m, (int)M->A.n, p->L, p->M + 1, M->ctx->sm_count);
    return a.off + 256;
}

int dense_moments(cmsvd_matrix* M, const cmsvd_params* p, const double2* quad, int Mk, const double* X, int64_t ldx,
                  double* S, int64_t lds, Arena& ws) {
    cmsvd_context* ctx = M->ctx;
    cudaStream_t s = ctx->s;
    const int64_t m = M->A.m;
    const int n = (int)M->A.n, L = p->L;
    if (M->A.n > 1024) { set_error("DENSE solver needs n <= 1024 (n = %lld)", (long long)M->A.n); return CMSVD_NOT_SUPPORTED; }
    if (lds != (int64_t)L * Mk) { set_error("DENSE solver writes S with leading dimension L (M + 1)"); return CMSVD_INVALID_ARG; }
    DenseBufs b;
    dense_alloc(b, ws, m, n, L, Mk, ctx->sm_count);
    if (!ws.fits()) { set_error("workspace too small"); return CMSVD_WORKSPACE_TOO_SMALL; }
    // H = A^T A, DD_BLOCK columns at a time
    for (int j0 = 0; j0 < n; j0 += DD_BLOCK) {
        const int bw = n - j0 < DD_BLOCK ? n - j0 : DD_BLOCK;
        CM_CUDA(cudaMemsetAsync(b.D, 0, sizeof(double) * (size_t)m * bw, s));
        {
            ProfScope ps(CMSVD_PROF_DIRECT, s, 12.0 * M->A.nnz + 8.0 * m * bw, 0.0);
            k_expand_cols<<<ctx->sm_count * 8, 256, 0, s>>>(M->A.rowptr, M->A.colidx, M->A.vals, m, j0, bw, b.D);
            CM_LAUNCH();
        }
        CM_TRY(spmm(M->At, bw, b.D, bw, b.H + j0, n, s));
    }
    // H = W diag(lambda) W^T: H V = Xc, lambda_j = ||Xc_j||, W = V (column-major)
    CM_TRY(jacobi_svd(b.H, n, n, 0, b.Xc, b.V, b.sv, b.perm, b.ints, ctx, 0.0, b.jctl));
    {
        ProfScope ps(CMSVD_PROF_DIRECT, s, 8.0 * n * (1.0 + Mk), (double)n * (p->N / 2) * (12.0 + 8.0 * Mk));
        k_dense_coef<<<(n + 127) / 128, 128, 0, s>>>(b.sv, n, quad, p->N / 2, Mk, p->ell, b.coef);
        CM_LAUNCH();
    }
    // Z = W^T X: the column-major V read as a row-major matrix is W^T
    CM_TRY(gemm_nn(b.V, n, X, ldx, b.Z, L, n, n, L, s));
    {
        ProfScope ps(CMSVD_PROF_DIRECT, s, 16.0 * n * L * Mk, (double)n * L * Mk);
        k_dense_scale<<<ctx->sm_count * 4, 256, 0, s>>>(b.Z, b.coef, n, L, Mk, b.Wall);
        CM_LAUNCH();
    }
    // S = W Wall = (W^T)^T Wall
    CM_TRY(gram(b.V, n, n, b.Wall, (int64_t)L * Mk, L * Mk, n, S, b.part, b.pcap, ctx->sm_count, s));
    return CMSVD_OK;
}

}  // namespace cmsvd

