// CSR storage of A and A^T: upload, validation, rounding of the values to the storage
// precision, the transpose, and the FP32 / bf16 copies the mixed-precision SpMM streams.
// The SpMM kernels themselves are in spmm.cu.
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

cmsvd_context*& current_ctx() {
    static thread_local cmsvd_context* c = nullptr;
    return c;
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
    A->sm_count = ctx->sm_count;
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
    if (A->vals_lo) cudaFree(A->vals_lo);
    if (A->vals_h) cudaFree(A->vals_h);
    if (A->row_order) cudaFree(A->row_order);
    A->rowptr = nullptr; A->colidx = nullptr; A->vals = nullptr; A->vals_f = nullptr; A->vals_lo = nullptr;
    A->vals_h = nullptr; A->row_order = nullptr;
}

// FP32 copy of the values (round to nearest); flags a value that is not FP32-exact.
__global__ void k_to_fp32(const double* __restrict__ x, int64_t n, float* __restrict__ y, int* __restrict__ inexact) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float f = __double2float_rn(x[i]);
        y[i] = f;
        bad |= (double)f != x[i];
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(inexact, 1);
}

// lo = x - hi, rounded to FP32: x = hi + lo to within 2^-48 |x|
__global__ void k_fp32_lo(const double* __restrict__ x, const float* __restrict__ hi, int64_t n, float* __restrict__ lo) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        lo[i] = __double2float_rn(x[i] - (double)hi[i]);
}

// FP32 copies of the values of A and A^T, made once per matrix. When some value is not
// FP32-exact (FP64 storage of general values), the remainders lo = a - fl32(a) are kept too:
// the double-float SpMM then multiplies by hi + lo.
int csr_make_fp32(cmsvd_matrix* M) {
    cmsvd_context* ctx = M->ctx;
    Csr* mats[2] = {&M->A, &M->At};
    for (Csr* c : mats) {
        if (c->vals_f) continue;
        CM_CUDA(cudaMalloc(&c->vals_f, sizeof(float) * (c->nnz > 0 ? c->nnz : 1)));
        int* flag = nullptr;
        CM_CUDA(cudaMalloc(&flag, sizeof(int)));
        int st = CMSVD_OK;
        auto chk = [&](cudaError_t e, const char* w) { if (e != cudaSuccess && st == CMSVD_OK) st = cuda_fail(e, w, __FILE__, __LINE__); };
        chk(cudaMemsetAsync(flag, 0, sizeof(int), ctx->s), "memset");
        if (c->nnz > 0) {
            k_to_fp32<<<ctx->sm_count * 4, 256, 0, ctx->s>>>(c->vals, c->nnz, c->vals_f, flag);
            note_launch();
            chk(cudaGetLastError(), "k_to_fp32");
        }
        chk(cudaMemcpyAsync(ctx->pinned, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s), "copy flag");
        chk(cudaStreamSynchronize(ctx->s), "sync");
        cudaFree(flag);
        if (st != CMSVD_OK) return st;
        c->f32_exact = ctx->pinned[0] ? 0 : 1;
        if (!c->f32_exact) {
            CM_CUDA(cudaMalloc(&c->vals_lo, sizeof(float) * c->nnz));
            k_fp32_lo<<<ctx->sm_count * 4, 256, 0, ctx->s>>>(c->vals, c->vals_f, c->nnz, c->vals_lo);
            CM_LAUNCH();
        }
    }
    return CMSVD_OK;
}

// Rounds the FP64 values to the storage precision in place (FP32 or bf16, round to nearest
// even) and, for bf16, keeps the 16-bit patterns the mixed-precision SpMM streams.
__global__ void k_round_storage(double* __restrict__ v, int64_t n, int storage, uint16_t* __restrict__ h,
                                int* __restrict__ overflow) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float f = __double2float_rn(v[i]);
        if (!isfinite(f)) atomicOr(overflow, 1);
        if (storage == CMSVD_STORE_FP32) {
            v[i] = (double)f;
        } else {
            uint32_t u = __float_as_uint(f);
            if ((u & 0x7f800000u) != 0x7f800000u) u += 0x7fffu + ((u >> 16) & 1u);   // round to nearest even
            const uint16_t b = (uint16_t)(u >> 16);
            h[i] = b;
            v[i] = (double)__uint_as_float((uint32_t)b << 16);
        }
    }
}

int csr_round_storage(cmsvd_context* ctx, Csr* A, int storage) {
    A->storage = storage;
    if (storage == CMSVD_STORE_FP64 || A->nnz == 0) return CMSVD_OK;
    if (storage == CMSVD_STORE_BF16) CM_CUDA(cudaMalloc(&A->vals_h, sizeof(uint16_t) * A->nnz));
    int* flag = nullptr;
    CM_CUDA(cudaMalloc(&flag, sizeof(int)));
    int st = CMSVD_OK;
    auto chk = [&](cudaError_t e, const char* w) { if (e != cudaSuccess && st == CMSVD_OK) st = cuda_fail(e, w, __FILE__, __LINE__); };
    chk(cudaMemsetAsync(flag, 0, sizeof(int), ctx->s), "memset");
    k_round_storage<<<ctx->sm_count * 4, 256, 0, ctx->s>>>(A->vals, A->nnz, storage, A->vals_h, flag);
    note_launch();
    chk(cudaGetLastError(), "k_round_storage");
    chk(cudaMemcpyAsync(ctx->pinned, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s), "copy flag");
    chk(cudaStreamSynchronize(ctx->s), "sync");
    cudaFree(flag);
    if (st != CMSVD_OK) return st;
    if (ctx->pinned[0]) {
        set_error("a value is outside the range of the storage precision");
        return CMSVD_INVALID_MATRIX;
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

}  // namespace cmsvd
