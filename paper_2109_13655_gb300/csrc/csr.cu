// CSR storage of A and A^T, validation, and the SpMM Y = A X that every
// shifted solve (Alg. 1 steps 1-2, as H X = A^T (A X)) and step 4 (A V~) use.
#include "internal.cuh"
#include <cub/device/device_radix_sort.cuh>
#include <cstdarg>
#include <cstdio>

namespace cmsvd {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char* last_error() { return g_err; }

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? CMSVD_OUT_OF_MEMORY : CMSVD_CUDA_ERROR;
}

// ----------------------------------------------------------------------------- profiler
Profiler& prof() {
    static thread_local Profiler p;
    return p;
}

void prof_reset(bool timing) {
    Profiler& p = prof();
    for (int i = 0; i < p.nrec; ++i) {
        cudaEventDestroy(p.recs[i].e0);
        cudaEventDestroy(p.recs[i].e1);
    }
    p.nrec = 0;
    p.launches = 0;
    p.captured = 0;
    p.capture_depth = 0;
    p.timing = timing;
}

ProfScope::ProfScope(int cls, cudaStream_t s, double bytes, double flops, int64_t launches) {
    Profiler& p = prof();
    if (!p.timing || p.capture_depth > 0 || p.nrec >= 4096) return;
    Profiler::Rec& r = p.recs[p.nrec];
    if (cudaEventCreate(&r.e0) != cudaSuccess) return;
    if (cudaEventCreate(&r.e1) != cudaSuccess) { cudaEventDestroy(r.e0); return; }
    r.cls = cls;
    r.bytes = bytes;
    r.flops = flops;
    r.launches = launches;
    cudaEventRecord(r.e0, s);
    idx = p.nrec++;
    stream_ = s;
}

ProfScope::~ProfScope() {
    if (idx >= 0) cudaEventRecord(prof().recs[idx].e1, stream_);
}

void prof_collect(cmsvd_stats* st) {
    Profiler& p = prof();
    st->kernel_launches = p.launches;
    for (int i = 0; i < p.nrec; ++i) {
        const Profiler::Rec& r = p.recs[i];
        float ms = 0.f;
        if (cudaEventSynchronize(r.e1) == cudaSuccess && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
            st->prof_ms[r.cls] += ms;
            st->prof_launches[r.cls] += r.launches;
            st->prof_bytes[r.cls] += r.bytes;
            st->prof_flops[r.cls] += r.flops;
        }
    }
    prof_reset(false);
}

static int grid_for(int64_t work, int per_block, int cap) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// ----------------------------------------------------------------------------- validation
// bad bits: 1 rowptr range, 2 column out of range, 4 columns not strictly increasing,
// 8 non-finite value, 16 rowptr[0] != 0 or rowptr[m] != nnz
__global__ void k_validate(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                           const double* __restrict__ vals, int64_t m, int64_t n, int64_t nnz, int* bad) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0 && (rowptr[0] != 0 || rowptr[m] != nnz)) atomicOr(bad, 16);
    int local = 0;
    for (int64_t i = i0; i < m; i += stride) {
        int64_t s = rowptr[i], e = rowptr[i + 1];
        if (s < 0 || e < s || e > nnz) { local |= 1; continue; }
        int32_t prev = -1;
        for (int64_t p = s; p < e; ++p) {
            int32_t c = colidx[p];
            if (c < 0 || c >= n) local |= 2;
            if (c <= prev) local |= 4;
            prev = c;
            if (!isfinite(vals[p])) local |= 8;
        }
    }
    if (local) atomicOr(bad, local);
}

__global__ void k_max_row(const int64_t* __restrict__ rowptr, int64_t m, unsigned long long* __restrict__ out) {
    unsigned long long best = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long len = (unsigned long long)(rowptr[r + 1] - rowptr[r]);
        best = len > best ? len : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

__global__ void k_first_col(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int64_t m,
                            int32_t* __restrict__ key, int32_t* __restrict__ idx) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        key[r] = rowptr[r + 1] > rowptr[r] ? colidx[rowptr[r]] : 0x7fffffff;
        idx[r] = (int32_t)r;
    }
}

// SpMM processing order: rows sorted (stably) by their first column, so that rows that
// gather the same rows of X run close together and find them in L2 (a permuted block
// matrix otherwise re-reads X from DRAM for every row). Each row's own sum is unchanged,
// so the SpMM result is bitwise the same in any order.
static int csr_row_order(cmsvd_context* ctx, Csr* A) {
    if (A->m <= 1 || A->m >= ((int64_t)1 << 31)) return CMSVD_OK;
    const int m = (int)A->m;
    int32_t *key = nullptr, *key_out = nullptr, *idx = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    int st = CMSVD_OK;
    auto chk = [&](cudaError_t e, const char* w) { if (e != cudaSuccess && st == CMSVD_OK) st = cuda_fail(e, w, __FILE__, __LINE__); };
    chk(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key, key_out, idx, A->row_order, m, 0, 31, ctx->s),
        "row order sort size");
    if (st == CMSVD_OK && (cudaMalloc(&key, sizeof(int32_t) * m) != cudaSuccess ||
                           cudaMalloc(&key_out, sizeof(int32_t) * m) != cudaSuccess ||
                           cudaMalloc(&idx, sizeof(int32_t) * m) != cudaSuccess ||
                           cudaMalloc(&A->row_order, sizeof(int32_t) * m) != cudaSuccess ||
                           cudaMalloc(&tmp, tmp_bytes > 0 ? tmp_bytes : 1) != cudaSuccess)) {
        cudaGetLastError();
        set_error("out of device memory for the SpMM row order");
        st = CMSVD_OUT_OF_MEMORY;
    }
    if (st == CMSVD_OK) {
        k_first_col<<<grid_for(A->m, 256, ctx->sm_count * 8), 256, 0, ctx->s>>>(A->rowptr, A->colidx, A->m, key, idx);
        chk(cudaGetLastError(), "k_first_col");
        chk(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, key, key_out, idx, A->row_order, m, 0, 31, ctx->s),
            "row order sort");
        chk(cudaStreamSynchronize(ctx->s), "sync");
    }
    for (void* ptr : {(void*)key, (void*)key_out, (void*)idx, tmp})
        if (ptr) cudaFree(ptr);
    if (st != CMSVD_OK && A->row_order) {
        cudaFree(A->row_order);
        A->row_order = nullptr;
    }
    return st;
}

// Longest row of a CSR already on the device (sets A->max_row), and the SpMM row order.
static int csr_row_stats(cmsvd_context* ctx, Csr* A) {
    unsigned long long* d = nullptr;
    CM_CUDA(cudaMalloc(&d, sizeof(unsigned long long)));
    int st = CMSVD_OK;
    auto chk = [&](cudaError_t e, const char* w) { if (e != cudaSuccess && st == CMSVD_OK) st = cuda_fail(e, w, __FILE__, __LINE__); };
    chk(cudaMemsetAsync(d, 0, sizeof(unsigned long long), ctx->s), "memset");
    k_max_row<<<grid_for(A->m, 256, ctx->sm_count * 8), 256, 0, ctx->s>>>(A->rowptr, A->m, d);
    chk(cudaGetLastError(), "k_max_row");
    unsigned long long h = 0;
    chk(cudaMemcpyAsync(ctx->pinned, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->s), "copy");
    chk(cudaStreamSynchronize(ctx->s), "sync");
    memcpy(&h, ctx->pinned, sizeof(h));
    cudaFree(d);
    A->max_row = (int64_t)h;
    if (st == CMSVD_OK) st = csr_row_order(ctx, A);
    return st;
}

int csr_upload_validate(cmsvd_context* ctx, int64_t m, int64_t n, int64_t nnz, const int64_t* rowptr,
                        const int32_t* colidx, const double* vals, int where, Csr* out) {
    cudaStream_t s = ctx->s;
    Csr A;
    A.m = m; A.n = n; A.nnz = nnz;
    CM_CUDA(cudaMalloc(&A.rowptr, sizeof(int64_t) * (m + 1)));
    if (cudaMalloc(&A.colidx, sizeof(int32_t) * (nnz > 0 ? nnz : 1)) != cudaSuccess ||
        cudaMalloc(&A.vals, sizeof(double) * (nnz > 0 ? nnz : 1)) != cudaSuccess) {
        csr_free(&A);
        set_error("out of device memory for a CSR with %lld nonzeros", (long long)nnz);
        return CMSVD_OUT_OF_MEMORY;
    }
    cudaMemcpyKind kind = where ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int st = CMSVD_OK;
    auto chk = [&](cudaError_t e, const char* w) { if (e != cudaSuccess && st == CMSVD_OK) st = cuda_fail(e, w, __FILE__, __LINE__); };
    chk(cudaMemcpyAsync(A.rowptr, rowptr, sizeof(int64_t) * (m + 1), kind, s), "copy rowptr");
    if (nnz > 0) {
        chk(cudaMemcpyAsync(A.colidx, colidx, sizeof(int32_t) * nnz, kind, s), "copy colidx");
        chk(cudaMemcpyAsync(A.vals, vals, sizeof(double) * nnz, kind, s), "copy vals");
    }
    int* bad_d = nullptr;
    chk(cudaMalloc(&bad_d, sizeof(int)), "alloc flag");
    if (st == CMSVD_OK) {
        chk(cudaMemsetAsync(bad_d, 0, sizeof(int), s), "memset");
        k_validate<<<grid_for(m, 256, ctx->sm_count * 8), 256, 0, s>>>(A.rowptr, A.colidx, A.vals, m, n, nnz, bad_d);
        chk(cudaGetLastError(), "k_validate");
        chk(cudaMemcpyAsync(ctx->pinned, bad_d, sizeof(int), cudaMemcpyDeviceToHost, s), "copy flag");
        chk(cudaStreamSynchronize(s), "sync");
    }
    if (bad_d) cudaFree(bad_d);
    if (st != CMSVD_OK) { csr_free(&A); return st; }
    int bad = ctx->pinned[0];
    if (bad) {
        csr_free(&A);
        set_error("invalid CSR (flags 0x%x: 1 row pointer range, 2 column index range, 4 unsorted or duplicate "
                  "columns, 8 non-finite value, 16 rowptr ends)", bad);
        return CMSVD_INVALID_MATRIX;
    }
    st = csr_row_stats(ctx, &A);
    if (st != CMSVD_OK) { csr_free(&A); return st; }
    *out = A;
    return CMSVD_OK;
}

void csr_free(Csr* A) {
    if (A->rowptr) cudaFree(A->rowptr);
    if (A->colidx) cudaFree(A->colidx);
    if (A->vals) cudaFree(A->vals);
    if (A->vals_f) cudaFree(A->vals_f);
    if (A->row_order) cudaFree(A->row_order);
    A->rowptr = nullptr; A->colidx = nullptr; A->vals = nullptr; A->vals_f = nullptr; A->row_order = nullptr;
}

__global__ void k_to_fp32(const double* __restrict__ x, int64_t n, float* __restrict__ y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = (float)x[i];
}

// FP32 copies of the values of A and A^T (round to nearest), made once per matrix.
int csr_make_fp32(cmsvd_matrix* M) {
    cmsvd_context* ctx = M->ctx;
    Csr* mats[2] = {&M->A, &M->At};
    for (Csr* c : mats) {
        if (c->vals_f) continue;
        CM_CUDA(cudaMalloc(&c->vals_f, sizeof(float) * (c->nnz > 0 ? c->nnz : 1)));
        if (c->nnz > 0) {
            k_to_fp32<<<ctx->sm_count * 4, 256, 0, ctx->s>>>(c->vals, c->nnz, c->vals_f);
            CM_LAUNCH();
        }
    }
    return CMSVD_OK;
}

// ----------------------------------------------------------------------------- transpose
__global__ void k_col_count(const int32_t* __restrict__ colidx, int64_t nnz, unsigned long long* counts) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride)
        atomicAdd(&counts[colidx[p] + 1], 1ull);
}

// In-place inclusive scan of len int64 values with one block of 1024 threads.
__global__ void k_scan_inclusive(int64_t* v, int64_t len) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    int64_t chunk = (len + 1023) / 1024;
    int64_t lo = t * chunk, hi = lo + chunk < len ? lo + chunk : len;
    int64_t sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += v[i];
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int64_t add = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    int64_t run = t ? part[t - 1] : 0;
    for (int64_t i = lo; i < hi; ++i) { run += v[i]; v[i] = run; }
}

// Row index of every nonzero (int32; m < 2^31).
__global__ void k_row_ids(const int64_t* __restrict__ rowptr, int64_t m, int32_t* __restrict__ rid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) rid[p] = (int32_t)i;
}

// A^T entries in (column, row) order from the stable column sort of A's nonzeros.
__global__ void k_gather_t(const int32_t* __restrict__ order, const int32_t* __restrict__ rid,
                           const double* __restrict__ vals, int64_t nnz, int32_t* __restrict__ tcol,
                           double* __restrict__ tval) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
        const int32_t o = order[p];
        tcol[p] = rid[o];
        tval[p] = vals[o];
    }
}

__global__ void k_iota(int32_t* __restrict__ x, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] = (int32_t)i;
}

// The scatter order inside a column depends on atomics; sorting each column by
// row index makes the transpose (and every SpMM with it) deterministic.

// A^T in CSR. Row pointers from per-column counts and a scan; the entries from a stable
// radix sort of A's nonzeros by column (A's storage order is row-major and row-sorted, so
// the rows of every column come out ascending). Deterministic, O(nnz) work per digit pass,
// whatever the row lengths of A^T.
int csr_transpose(cmsvd_context* ctx, const Csr& A, Csr* At) {
    cudaStream_t s = ctx->s;
    if (A.nnz >= ((int64_t)1 << 31) || A.m >= ((int64_t)1 << 31)) {
        set_error("the transpose supports fewer than 2^31 rows and nonzeros");
        return CMSVD_NOT_SUPPORTED;
    }
    const int nnz = (int)A.nnz;
    Csr T;
    T.m = A.n; T.n = A.m; T.nnz = A.nnz;
    CM_CUDA(cudaMalloc(&T.rowptr, sizeof(int64_t) * (T.m + 1)));
    if (cudaMalloc(&T.colidx, sizeof(int32_t) * (nnz > 0 ? nnz : 1)) != cudaSuccess ||
        cudaMalloc(&T.vals, sizeof(double) * (nnz > 0 ? nnz : 1)) != cudaSuccess) {
        csr_free(&T);
        set_error("out of device memory for the transpose");
        return CMSVD_OUT_OF_MEMORY;
    }
    int st = CMSVD_OK;
    auto chk = [&](cudaError_t e, const char* w) { if (e != cudaSuccess && st == CMSVD_OK) st = cuda_fail(e, w, __FILE__, __LINE__); };
    chk(cudaMemsetAsync(T.rowptr, 0, sizeof(int64_t) * (T.m + 1), s), "memset");
    const int gcap = ctx->sm_count * 8;
    k_col_count<<<grid_for(A.nnz, 256, gcap), 256, 0, s>>>(A.colidx, A.nnz, (unsigned long long*)T.rowptr);
    chk(cudaGetLastError(), "k_col_count");
    k_scan_inclusive<<<1, 1024, 0, s>>>(T.rowptr, T.m + 1);
    chk(cudaGetLastError(), "k_scan");
    if (nnz > 0 && st == CMSVD_OK) {
        int32_t *keys_out = nullptr, *idx_in = nullptr, *idx_out = nullptr, *rid = nullptr;
        void* tmp = nullptr;
        size_t tmp_bytes = 0;
        int end_bit = 1;
        while (end_bit < 31 && ((int64_t)1 << end_bit) < A.n) ++end_bit;
        chk(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, A.colidx, keys_out, idx_in, idx_out, nnz, 0, end_bit, s),
            "radix sort size");
        if (st == CMSVD_OK && (cudaMalloc(&keys_out, sizeof(int32_t) * nnz) != cudaSuccess ||
                               cudaMalloc(&idx_in, sizeof(int32_t) * nnz) != cudaSuccess ||
                               cudaMalloc(&idx_out, sizeof(int32_t) * nnz) != cudaSuccess ||
                               cudaMalloc(&rid, sizeof(int32_t) * nnz) != cudaSuccess ||
                               cudaMalloc(&tmp, tmp_bytes > 0 ? tmp_bytes : 1) != cudaSuccess)) {
            cudaGetLastError();
            set_error("out of device memory for the transpose sort");
            st = CMSVD_OUT_OF_MEMORY;
        }
        if (st == CMSVD_OK) {
            k_iota<<<grid_for(A.nnz, 256, gcap), 256, 0, s>>>(idx_in, A.nnz);
            chk(cudaGetLastError(), "k_iota");
            k_row_ids<<<grid_for(A.m, 256, gcap), 256, 0, s>>>(A.rowptr, A.m, rid);
            chk(cudaGetLastError(), "k_row_ids");
            chk(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, A.colidx, keys_out, idx_in, idx_out, nnz, 0, end_bit, s),
                "radix sort");
            k_gather_t<<<grid_for(A.nnz, 256, gcap), 256, 0, s>>>(idx_out, rid, A.vals, A.nnz, T.colidx, T.vals);
            chk(cudaGetLastError(), "k_gather_t");
        }
        chk(cudaStreamSynchronize(s), "sync");
        for (void* ptr : {(void*)keys_out, (void*)idx_in, (void*)idx_out, (void*)rid, tmp})
            if (ptr) cudaFree(ptr);
    }
    chk(cudaStreamSynchronize(s), "sync");
    if (st == CMSVD_OK) st = csr_row_stats(ctx, &T);
    if (st != CMSVD_OK) { csr_free(&T); return st; }
    *At = T;
    return CMSVD_OK;
}

// ----------------------------------------------------------------------------- SpMM
// One group of LPR lanes per row; lane l owns columns l, l+LPR, ... of the
// row-major L-column block. The row's (col, val) pairs are loaded cooperatively
// and broadcast with shuffles, so every nonzero reads one contiguous L-vector of
// X. Each output element is summed in the row's storage order (deterministic).
__device__ __forceinline__ double fma_rn_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// One chunk of up to LPR nonzeros of a row, broadcast from the lanes that loaded them:
// the X rows of SPMM_ILP nonzeros are gathered before their multiply-adds, so that many
// gathers are in flight (a gather whose address comes from a shuffle otherwise waits for
// the previous multiply-add). The multiply-adds stay in the row's storage order.
constexpr int SPMM_ILP = 8;
template <typename T, int LPR, int CPL>
__device__ __forceinline__ void spmm_chunk(unsigned mask, int32_t mc, T mv, int cnt, const T* __restrict__ X,
                                           int64_t ldx, int c0, int lane, int L, T (&acc)[CPL]) {
    int k0 = 0;
    for (; k0 + SPMM_ILP <= cnt; k0 += SPMM_ILP) {   // full groups: gathers first, then the multiply-adds
        T xv[SPMM_ILP][CPL];
        T vv[SPMM_ILP];
#pragma unroll
        for (int u = 0; u < SPMM_ILP; ++u) {
            const int32_t col = __shfl_sync(mask, mc, k0 + u, LPR);
            vv[u] = __shfl_sync(mask, mv, k0 + u, LPR);
            const T* xr = X + (int64_t)col * ldx + c0 + lane;
#pragma unroll
            for (int q = 0; q < CPL; ++q) xv[u][q] = c0 + lane + q * LPR < L ? __ldg(xr + q * LPR) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < SPMM_ILP; ++u)
#pragma unroll
            for (int q = 0; q < CPL; ++q)
                if (c0 + lane + q * LPR < L) acc[q] = fma_rn_t(vv[u], xv[u][q], acc[q]);
    }
    for (; k0 < cnt; ++k0) {                          // the rest (short rows take only this path)
        const int32_t col = __shfl_sync(mask, mc, k0, LPR);
        const T v = __shfl_sync(mask, mv, k0, LPR);
        const T* xr = X + (int64_t)col * ldx + c0 + lane;
#pragma unroll
        for (int q = 0; q < CPL; ++q)
            if (c0 + lane + q * LPR < L) acc[q] = fma_rn_t(v, __ldg(xr + q * LPR), acc[q]);
    }
}

template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(256) k_spmm(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                              const T* __restrict__ vals, int64_t rows, int L,
                                              const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                              int64_t ldy, const int32_t* __restrict__ order) {
    const int lane = threadIdx.x % LPR;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / LPR;
    const unsigned mask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << ((threadIdx.x & 31) / LPR * LPR));
    for (int64_t rr = group; rr < rows; rr += ngroups) {
        const int64_t r = order ? (int64_t)order[rr] : rr;
        const int64_t s = rowptr[r], e = rowptr[r + 1];
        for (int c0 = 0; c0 < L; c0 += LPR * CPL) {
            T acc[CPL];
#pragma unroll
            for (int q = 0; q < CPL; ++q) acc[q] = (T)0;
            for (int64_t p0 = s; p0 < e; p0 += LPR) {
                const int64_t p = p0 + lane;
                int32_t mc = 0;
                T mv = (T)0;
                if (p < e) { mc = colidx[p]; mv = vals[p]; }
                const int cnt = (int)((e - p0) < LPR ? (e - p0) : LPR);
                spmm_chunk<T, LPR, CPL>(mask, mc, mv, cnt, X, ldx, c0, lane, L, acc);
            }
#pragma unroll
            for (int q = 0; q < CPL; ++q)
                if (c0 + lane + q * LPR < L) Y[r * ldy + c0 + lane + q * LPR] = acc[q];
        }
    }
}

// Long rows (a few rows holding most nonzeros, e.g. the transpose of a matrix whose
// columns are image pixels): one CTA per row. Its 256 / LPR groups take contiguous,
// equal slices of the row, and their partial sums are added in slice order, so the
// result is deterministic (the summation order differs from k_spmm's).
template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(256) k_spmm_rowcta(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                                     const T* __restrict__ vals, int64_t rows, int L,
                                                     const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                                     int64_t ldy, const int32_t* __restrict__ order) {
    constexpr int G = 256 / LPR;
    __shared__ T part[G][LPR * CPL];
    const int lane = threadIdx.x % LPR, g = threadIdx.x / LPR;
    const unsigned mask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << ((threadIdx.x & 31) / LPR * LPR));
    for (int64_t rr = blockIdx.x; rr < rows; rr += gridDim.x) {
        const int64_t r = order ? (int64_t)order[rr] : rr;
        const int64_t rs = rowptr[r], re = rowptr[r + 1];
        const int64_t slice = (re - rs + G - 1) / G;
        const int64_t s = rs + g * slice < re ? rs + g * slice : re;
        const int64_t e = s + slice < re ? s + slice : re;
        for (int c0 = 0; c0 < L; c0 += LPR * CPL) {
            T acc[CPL];
#pragma unroll
            for (int q = 0; q < CPL; ++q) acc[q] = (T)0;
            for (int64_t p0 = s; p0 < e; p0 += LPR) {
                const int64_t p = p0 + lane;
                int32_t mc = 0;
                T mv = (T)0;
                if (p < e) { mc = colidx[p]; mv = vals[p]; }
                const int cnt = (int)((e - p0) < LPR ? (e - p0) : LPR);
                spmm_chunk<T, LPR, CPL>(mask, mc, mv, cnt, X, ldx, c0, lane, L, acc);
            }
#pragma unroll
            for (int q = 0; q < CPL; ++q) part[g][lane + q * LPR] = acc[q];
            __syncthreads();
            for (int c = threadIdx.x; c < LPR * CPL; c += blockDim.x) {
                if (c0 + c < L) {
                    T sum = part[0][c];
                    for (int h = 1; h < G; ++h) sum += part[h][c];
                    Y[r * ldy + c0 + c] = sum;
                }
            }
            __syncthreads();
        }
    }
}

template <typename T>
static int spmm_t(const Csr& A, const T* vals, int L, const T* X, int64_t ldx, T* Y, int64_t ldy, cudaStream_t s) {
    if (A.m == 0 || L <= 0) return CMSVD_OK;
    // compulsory traffic: A (values, indices, row pointers), X once, Y once
    const double e = (double)sizeof(T);
    ProfScope ps(CMSVD_PROF_SPMM, s, (e + 4.0) * A.nnz + 8.0 * (A.m + 1) + e * L * (A.n + A.m), 2.0 * A.nnz * L);
    const int dev_sms = 152;
    if (A.max_row > 2048) {
        const unsigned grid = (unsigned)(A.m < dev_sms * 8 ? A.m : dev_sms * 8);
        if (L <= 8) k_spmm_rowcta<T, 8, 1><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, vals, A.m, L, X, ldx, Y, ldy, A.row_order);
        else if (L <= 16) k_spmm_rowcta<T, 16, 1><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, vals, A.m, L, X, ldx, Y, ldy, A.row_order);
        else if (L <= 32) k_spmm_rowcta<T, 32, 1><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, vals, A.m, L, X, ldx, Y, ldy, A.row_order);
        else k_spmm_rowcta<T, 32, 4><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, vals, A.m, L, X, ldx, Y, ldy, A.row_order);
        CM_LAUNCH();
        return CMSVD_OK;
    }
    if (L <= 8) {
        k_spmm<T, 8, 1><<<grid_for(A.m, 256 / 8, dev_sms * 32), 256, 0, s>>>(A.rowptr, A.colidx, vals, A.m, L, X, ldx, Y, ldy, A.row_order);
    } else if (L <= 16) {
        k_spmm<T, 16, 1><<<grid_for(A.m, 256 / 16, dev_sms * 32), 256, 0, s>>>(A.rowptr, A.colidx, vals, A.m, L, X, ldx, Y, ldy, A.row_order);
    } else if (L <= 32) {
        k_spmm<T, 32, 1><<<grid_for(A.m, 8, dev_sms * 32), 256, 0, s>>>(A.rowptr, A.colidx, vals, A.m, L, X, ldx, Y, ldy, A.row_order);
    } else {
        k_spmm<T, 32, 4><<<grid_for(A.m, 8, dev_sms * 32), 256, 0, s>>>(A.rowptr, A.colidx, vals, A.m, L, X, ldx, Y, ldy, A.row_order);
    }
    CM_LAUNCH();
    return CMSVD_OK;
}

int spmm(const Csr& A, int L, const double* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t s) {
    return spmm_t<double>(A, A.vals, L, X, ldx, Y, ldy, s);
}

int spmm(const Csr& A, int L, const float* X, int64_t ldx, float* Y, int64_t ldy, cudaStream_t s) {
    if (!A.vals_f) { set_error("FP32 values of A were not made"); return CMSVD_INVALID_ARG; }
    return spmm_t<float>(A, A.vals_f, L, X, ldx, Y, ldy, s);
}

}  // namespace cmsvd
