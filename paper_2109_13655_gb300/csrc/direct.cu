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
// the device.
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
    for (int i = lane; i < s; i += 32) {
        const double lam = H[i * s + i];
        double f = 0.0;
        for (int m = 0; m < a.Mk; ++m) coef[m * s + i] = 0.0;
        for (int j = 0; j < a.J; ++j) {
            const double2 sh = a.quad[3 * j], w = a.quad[3 * j + 1], sc = a.quad[3 * j + 2];
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
            for (int m = 0; m < a.Mk; ++m) {
                coef[m * s + i] += 2.0 * gr;
                const double nr = gr * sc.x - gi * sc.y, ni = gr * sc.y + gi * sc.x;
                gr = nr;
                gi = ni;
            }
        }
        double fp = 1.0;
        for (int e = 1; e < a.ell; ++e) fp *= f;
        for (int m = 0; m < a.Mk; ++m) coef[m * s + i] *= fp;
    }
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

}  // namespace cmsvd
