// FP64-accurate tall-skinny Gram (G = X^T Y) and product (Z = X W) from exact BF16 tensor-core
// products: the rank truncation (Alg. 1 step 3) and qr(A V~) (step 4) are built on these two
// products, and GB300's FP64 pipe issues 2 FMAs per clock per SM against its BF16 tensor cores'
// ~900.
//
// Splitting (an Ozaki-type scheme): every operand value is written as
//   x = s 2^e sum_{p=1..S} d_p 2^{-7p} + r,   d_p in [0, 127] (with the sign s of x), |r| < 2^(e-56),
// with S = 8 slices of 7 bits and a power-of-two scale 2^e > |x| per column (Gram) or per row /
// column (product). A slice value d is an integer below 128, so it is exact in bf16, every product
// of two slices is an integer below 2^14, and any sum of at most 1024 such products is an integer
// below 2^24: the FP32 accumulation of the tensor cores is then exact whatever its order. The
// Gram forms one GEMM output per slice pair and block of 1024 rows (a batched GEMM over the
// blocks with K = 1024); the product stacks up to 1024 / c1 slice pairs of a level along the
// contraction. The exact outputs are added per level k = p + q (scale 2^(-7k)) in integer
// arithmetic and the level sums combined into the FP64 result, scaled by 2^(e_i + f_j). Pairs with p + q > S + 1 are dropped: per
// product their sum is below 2^-53 of 2^(e_i + f_j). With the truncation of the operands to 56
// bits below their scales, each emulated product is within a few 2^-53 of 2^(e_i + f_j), that is
// of the products of the largest entries sharing the scales: FP64 accuracy for operands whose
// entries are of one magnitude within a row or column (orthogonalized blocks), and the accuracy
// class of an FP64 Gram of this length (sqrt(n) u sum |x||y|) in general.
//
// The slice products are plain BF16 GEMMs with FP32 outputs and run on cuBLAS; slicing and the
// FP64 epilogue are this file's kernels.
#include "internal.cuh"
#include "ozaki_math.cuh"
#include <cublas_v2.h>
#include <climits>

namespace cmsvd {

constexpr int OZ_KMAX = 1024;    // products per exact FP32 sum
constexpr int OZ_CHUNK = 1024;   // Gram: rows per block (one slice pair of a block: 1024 products)
constexpr int OZ_PAIRS = 36;     // slice pairs (p, q), p + q <= S + 1 (levels 2..9)
static_assert(OZ_S == 8 && OZ_BITS == 7, "the epilogues combine levels 2..5 and 6..9");

// ----------------------------------------------------------------------------- scales
// ilogb of the largest |x| of each column (cols of an n x c row-major block) / each row
// (oz_ilogb: from the exponent field).
__global__ void k_oz_col_exp(const double* __restrict__ X, int64_t ld, int64_t n, int c, int* __restrict__ ex) {
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
        int best = INT_MIN;
        for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
            const double v = X[i * ld + j];
            if ((__double_as_longlong(v) << 1) != 0) best = max(best, oz_ilogb(v));
        }
        if (best != INT_MIN) atomicMax(ex + j, best);
    }
}

__global__ void k_oz_row_exp(const double* __restrict__ X, int64_t ld, int64_t n, int c, int* __restrict__ ex) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) / 32) {
        int best = INT_MIN;
        for (int j = lane; j < c; j += 32) {
            const double v = X[i * ld + j];
            if ((__double_as_longlong(v) << 1) != 0) best = max(best, oz_ilogb(v));
        }
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) ex[i] = best;
    }
}

// scale exponents are initialised to OZ_NONE (all-zero column or row)
constexpr int OZ_NONE = (int)0x80808080;
__device__ __forceinline__ int oz_e(int e) { return e == OZ_NONE || e == INT_MIN ? 0 : e; }
__device__ __forceinline__ int oz_shift(int e) { return e == OZ_NONE || e == INT_MIN ? 0 : e + 1; }


// Gram operand: X (n x c row-major) -> per block b of OZ_CHUNK rows, S slices of cp x OZ_CHUNK
// column-major (ld cp, cp = c rounded up to 8: the pad entries are zero, and the GEMMs see
// 16-byte aligned operands), slice p at block position p in fw and at position S-1-p in rv
// (either may be null). One CTA row at a time (threads over columns).
__global__ void k_oz_slice_gram(const double* __restrict__ X, int64_t ld, int64_t n, int c, int cp,
                                const int* __restrict__ ex, __nv_bfloat16* __restrict__ fw, __nv_bfloat16* __restrict__ rv) {
    const int64_t bs = (int64_t)OZ_S * cp * OZ_CHUNK, ss = (int64_t)cp * OZ_CHUNK;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t b = i / OZ_CHUNK, il = i % OZ_CHUNK;
        for (int j = threadIdx.x; j < cp; j += blockDim.x) {
            float d[OZ_S];
            if (j < c) oz_slices(X[i * ld + j], oz_e(ex[j]), d);
            else {
#pragma unroll
                for (int p = 0; p < OZ_S; ++p) d[p] = 0.f;
            }
            const int64_t o = b * bs + il * cp + j;
#pragma unroll
            for (int p = 0; p < OZ_S; ++p) {
                const __nv_bfloat16 v = __float2bfloat16_rn(d[p]);
                if (fw) fw[o + p * ss] = v;
                if (rv) rv[o + (OZ_S - 1 - p) * ss] = v;
            }
        }
    }
}

// Product operands (c1p, c2p: c1, c2 rounded up to 8, pads zero). X (n x c1, row-major, row
// scale): column-major (S c1p) x n, ld S c1p, slice p of row i at rows p c1p .. p c1p + c1 - 1 of
// column i (one CTA row at a time). W (c1 x c2, row-major, column scale): S column-major
// c2p x c1p blocks (ld c2p), slice q at block S-1-q (reversed).
__global__ void k_oz_slice_rows(const double* __restrict__ X, int64_t ld, int64_t n, int c1, int c1p,
                                const int* __restrict__ ex, __nv_bfloat16* __restrict__ out) {
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        __nv_bfloat16* col = out + i * (int64_t)OZ_S * c1p;
        const int e = oz_e(ex[i]);
        for (int j = threadIdx.x; j < c1p; j += blockDim.x) {
            float d[OZ_S];
            if (j < c1) oz_slices(X[i * ld + j], e, d);
            else {
#pragma unroll
                for (int p = 0; p < OZ_S; ++p) d[p] = 0.f;
            }
#pragma unroll
            for (int p = 0; p < OZ_S; ++p) col[(int64_t)p * c1p + j] = __float2bfloat16_rn(d[p]);
        }
    }
}

__global__ void k_oz_slice_w(const double* __restrict__ W, int64_t ldw, int c1, int c2, int c1p, int c2p,
                             const int* __restrict__ ex, __nv_bfloat16* __restrict__ out) {
    const int64_t total = (int64_t)c1p * c2p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / c2p), l = (int)(e % c2p);
        float d[OZ_S];
        if (k < c1 && l < c2) oz_slices(W[(int64_t)k * ldw + l], oz_e(ex[l]), d);
        else {
#pragma unroll
            for (int q = 0; q < OZ_S; ++q) d[q] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < OZ_S; ++q)
            out[(int64_t)(OZ_S - 1 - q) * c2p * c1p + (int64_t)k * c2p + l] = __float2bfloat16_rn(d[q]);
    }
}

// ----------------------------------------------------------------------------- epilogues
// The FP32 slice-GEMM outputs are exact integers below 2^24 in magnitude. The epilogues add
// them in integer arithmetic (FP32 -> int32 conversions and integer adds run off the FP64
// pipe, which GB300 issues at 2 lanes per clock per SM) and convert once: the levels 2..5 and
// 6..9 are combined into two int64 sums on the scales 2^-35 and 2^-63,
//   th = sum_{k=2..5} s_k 2^(7 (5 - k)),   tl = sum_{k=6..9} s_k 2^(7 (9 - k)),
// each below 2^53 in magnitude for level sums |s_k| < 2^28, so that
// sum_k s_k 2^(-7 k) = th 2^-35 + tl 2^-63 is formed by one FMA of two exact doubles with a
// single rounding.
__device__ __forceinline__ double oz_combine(long long th, long long tl) {
    return __fma_rn((double)th, 0x1p-35, (double)tl * 0x1p-63);
}


// Gram, pass 1: P[part][j + k c1] = sum_lvl 2^(-7 lvl) sum_{pairs of lvl} sum_{b in part}
// C[pair][b][j + k c1] over a part of OZ_PART blocks of the current group (blockIdx.y); a level
// sum over a part has at most 8 x 8 terms below 2^24: |s_k| < 2^30.
constexpr int OZ_PART = 8;
__global__ void k_oz_gram_part(const float* __restrict__ C, int nb, int64_t cnt, double* __restrict__ P) {
    const int part = blockIdx.y;
    const int b0 = part * OZ_PART, b1 = b0 + OZ_PART < nb ? b0 + OZ_PART : nb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        long long th = 0, tl = 0;
#pragma unroll
        for (int lvl = 2; lvl <= OZ_S + 1; ++lvl) {
            long long sk = 0;
            for (int t = 0; t < lvl - 1; ++t) {
                const float* Cp = C + (int64_t)((lvl - 2) * (lvl - 1) / 2 + t) * nb * cnt;
                for (int b = b0; b < b1; ++b) sk += __float2int_rz(__ldcs(Cp + (int64_t)b * cnt + e));
            }
            if (lvl <= 5) th += sk << (OZ_BITS * (5 - lvl));
            else tl += sk << (OZ_BITS * (9 - lvl));
        }
        P[(int64_t)part * cnt + e] = oz_combine(th, tl);
    }
}

// Gram, pass 2: G[j][k] = 2^(ex_j + 1 + ey_k + 1) sum_part P[part][j + k c1p], parts in order.
__global__ void k_oz_gram_fin(const double* __restrict__ P, int nparts, int c1, int c2, int c1p, int64_t cep,
                              const int* __restrict__ ex, const int* __restrict__ ey, double* __restrict__ G, int64_t ldg) {
    const int64_t cnt = (int64_t)c1 * c2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % c1), k = (int)(e / c1);
        double v = 0.0;
        for (int q = 0; q < nparts; ++q) v += P[(int64_t)q * cep + j + (int64_t)k * c1p];
        G[(int64_t)j * ldg + k] = ldexp(v, oz_shift(ex[j]) + oz_shift(ey[k]));
    }
}

// Product: Z[i][l] = 2^(ex_i + 1 + fw_l + 1) sum_g 2^(-7 lvl_g) C[g][l + i c2p] over the ng GEMM
// outputs of a row block (a level has at most 8 outputs: |s_k| < 2^27), written once. One CTA
// row at a time.
struct OzLevels { int lvl[64]; };   // level of each GEMM output
__global__ void k_oz_gemm_epi(const float* __restrict__ C, int ng, OzLevels lv, int64_t n, int c2, int c2p,
                              const int* __restrict__ ex, const int* __restrict__ ew, double* __restrict__ Z, int64_t ldz) {
    const int64_t gs = n * c2p;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int si = oz_shift(ex[i]);
        for (int l = threadIdx.x; l < c2; l += blockDim.x) {
            long long th = 0, tl = 0;
            for (int g = 0; g < ng; ++g) {
                const int lvl = lv.lvl[g];
                const long long sk = __float2int_rz(__ldcs(C + (int64_t)g * gs + i * c2p + l));
                if (lvl <= 5) th += sk << (OZ_BITS * (5 - lvl));
                else tl += sk << (OZ_BITS * (9 - lvl));
            }
            Z[i * ldz + l] = oz_to_double(th, tl, si + oz_shift(ew[l]));
        }
    }
}

// ----------------------------------------------------------------------------- host
static int blas_ok(cublasStatus_t s, const char* what) {
    if (s == CUBLAS_STATUS_SUCCESS) return CMSVD_OK;
    set_error("%s failed (cuBLAS status %d)", what, (int)s);
    return s == CUBLAS_STATUS_ALLOC_FAILED ? CMSVD_OUT_OF_MEMORY : CMSVD_CUDA_ERROR;
}

static int oz_handle(cmsvd_context* ctx, cublasHandle_t* h) {
    if (!ctx->blas) {
        cublasHandle_t x = nullptr;
        CM_TRY(blas_ok(cublasCreate(&x), "cublasCreate"));
        ctx->blas = x;
    }
    *h = (cublasHandle_t)ctx->blas;
    CM_TRY(blas_ok(cublasSetStream(*h, ctx->s), "cublasSetStream"));
    return CMSVD_OK;
}

// Scratch kept by the context between calls (grown on demand).
static int oz_scratch(cmsvd_context* ctx, size_t bytes, char** out) {
    if (ctx->oz_bytes < bytes) {
        if (ctx->oz_buf) {
            CM_CUDA(cudaStreamSynchronize(ctx->s));
            cudaFree(ctx->oz_buf);
            ctx->oz_buf = nullptr;
            ctx->oz_bytes = 0;
        }
        CM_CUDA(cudaMalloc(&ctx->oz_buf, bytes));
        ctx->oz_bytes = bytes;
    }
    *out = (char*)ctx->oz_buf;
    return CMSVD_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool ozaki_applies(const cmsvd_context* ctx, int64_t n, int c1, int c2) {
    return ctx && ctx->dense_arith == 0 && n >= 16384 && c1 >= 32 && c2 >= 32 && c1 <= OZ_KMAX;
}

// G (c1 x c2, row-major, ldg) = X^T Y.
int gram_ozaki(cmsvd_context* ctx, const double* X, int64_t ldx, int c1, const double* Y, int64_t ldy, int c2,
               int64_t n, double* G, int64_t ldg) {
    cudaStream_t s = ctx->s;
    cublasHandle_t h;
    CM_TRY(oz_handle(ctx, &h));
    const int64_t nb = (n + OZ_CHUNK - 1) / OZ_CHUNK;
    const bool same = X == Y && c1 == c2 && ldx == ldy;
    const int c1p = (c1 + 7) / 8 * 8, c2p = (c2 + 7) / 8 * 8;
    const int64_t ce = (int64_t)c1p * c2p;   // GEMM outputs, padded
    // GEMM outputs of a group of blocks: about 1 GB of FP32 at a time, whole parts per group
    int64_t nbg = (int64_t)((1ll << 30) / (OZ_PAIRS * ce * 4)) / OZ_PART * OZ_PART;
    if (nbg < OZ_PART) nbg = OZ_PART;
    if (nbg > nb) nbg = nb;
    const int64_t ngroups = (nb + nbg - 1) / nbg, ppg = (nbg + OZ_PART - 1) / OZ_PART, nparts = ngroups * ppg;
    const size_t bx = align256((size_t)nb * OZ_S * c1p * OZ_CHUNK * 2);
    const size_t byr = align256((size_t)nb * OZ_S * c2p * OZ_CHUNK * 2);
    const size_t bc = align256((size_t)OZ_PAIRS * nbg * ce * 4);
    const size_t bp = align256((size_t)nparts * ce * 8);
    const size_t be = align256(sizeof(int) * (c1 + c2));
    char* buf = nullptr;
    CM_TRY(oz_scratch(ctx, bx + byr + bc + bp + be, &buf));
    __nv_bfloat16* xs = (__nv_bfloat16*)buf;
    __nv_bfloat16* ys = (__nv_bfloat16*)(buf + bx);      // reversed slice order (the B operand)
    float* Cb = (float*)(buf + bx + byr);
    double* Pp = (double*)(buf + bx + byr + bc);
    int* ex = (int*)(buf + bx + byr + bc + bp);
    int* ey = ex + c1;
    ProfScope ps(CMSVD_PROF_GRAM, s, 8.0 * n * (same ? c1 : c1 + c2) + 8.0 * c1 * c2,
                 2.0 * n * c1 * c2);
    // the rows past n in the last block must be zero slices; parts of a short last group stay 0
    if (n % OZ_CHUNK) {
        const int64_t b = nb - 1;
        CM_CUDA(cudaMemsetAsync(xs + b * (int64_t)OZ_S * c1p * OZ_CHUNK, 0, (size_t)OZ_S * c1p * OZ_CHUNK * 2, s));
        CM_CUDA(cudaMemsetAsync(ys + b * (int64_t)OZ_S * c2p * OZ_CHUNK, 0, (size_t)OZ_S * c2p * OZ_CHUNK * 2, s));
    }
    CM_CUDA(cudaMemsetAsync(Pp, 0, (size_t)nparts * ce * 8, s));
    CM_CUDA(cudaMemsetAsync(ex, 0x80, sizeof(int) * (c1 + c2), s));   // OZ_NONE, below any ilogb
    const int grid = ctx->sm_count * 4;
    k_oz_col_exp<<<grid, 256, 0, s>>>(X, ldx, n, c1, ex);
    CM_LAUNCH();
    if (same) {
        CM_CUDA(cudaMemcpyAsync(ey, ex, sizeof(int) * c1, cudaMemcpyDeviceToDevice, s));
        k_oz_slice_gram<<<ctx->sm_count * 8, 256, 0, s>>>(X, ldx, n, c1, c1p, ex, xs, ys);
        CM_LAUNCH();
    } else {
        k_oz_col_exp<<<grid, 256, 0, s>>>(Y, ldy, n, c2, ey);
        CM_LAUNCH();
        k_oz_slice_gram<<<ctx->sm_count * 8, 256, 0, s>>>(X, ldx, n, c1, c1p, ex, xs, nullptr);
        CM_LAUNCH();
        k_oz_slice_gram<<<ctx->sm_count * 8, 256, 0, s>>>(Y, ldy, n, c2, c2p, ey, nullptr, ys);
        CM_LAUNCH();
    }
    const float one = 1.f, zero = 0.f;
    for (int64_t g = 0; g < ngroups; ++g) {
        const int64_t b0 = g * nbg, cnt = nb - b0 < nbg ? nb - b0 : nbg;
        for (int lvl = 2; lvl <= OZ_S + 1; ++lvl) {
            const int pairs = lvl - 1;
            for (int t = 0; t < pairs; ++t) {
                // X slice t against Y slice pairs-1-t (reversed storage: block position S-pairs+t)
                const int pi = (lvl - 2) * (lvl - 1) / 2 + t;
                const __nv_bfloat16* A = xs + (b0 * OZ_S + t) * (int64_t)c1p * OZ_CHUNK;
                const __nv_bfloat16* Bm = ys + (b0 * OZ_S + OZ_S - pairs + t) * (int64_t)c2p * OZ_CHUNK;
                CM_TRY(blas_ok(cublasGemmStridedBatchedEx(h, CUBLAS_OP_N, CUBLAS_OP_T, c1p, c2p, OZ_CHUNK, &one,
                                                          A, CUDA_R_16BF, c1p, (int64_t)OZ_S * c1p * OZ_CHUNK,
                                                          Bm, CUDA_R_16BF, c2p, (int64_t)OZ_S * c2p * OZ_CHUNK, &zero,
                                                          Cb + (int64_t)pi * cnt * ce, CUDA_R_32F, c1p, ce, (int)cnt,
                                                          CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT),
                               "cublasGemmStridedBatchedEx (Gram slices)"));
            }
        }
        dim3 pg((unsigned)((ce + 255) / 256 < 64 ? (ce + 255) / 256 : 64), (unsigned)((cnt + OZ_PART - 1) / OZ_PART));
        k_oz_gram_part<<<pg, 256, 0, s>>>(Cb, (int)cnt, ce, Pp + g * ppg * ce);
        CM_LAUNCH();
    }
    k_oz_gram_fin<<<(int)((ce + 255) / 256 < ctx->sm_count * 4 ? (ce + 255) / 256 : ctx->sm_count * 4), 256, 0, s>>>(
        Pp, (int)nparts, c1, c2, c1p, ce, ex, ey, G, ldg);
    CM_LAUNCH();
    return CMSVD_OK;
}

// Z (n x c2, ldz) = X (n x c1, ldx) W (c1 x c2, ldw).
int gemm_ozaki(cmsvd_context* ctx, const double* X, int64_t ldx, const double* W, int64_t ldw, double* Z, int64_t ldz,
               int64_t n, int c1, int c2) {
    cudaStream_t s = ctx->s;
    cublasHandle_t h;
    CM_TRY(oz_handle(ctx, &h));
    const int c1p = (c1 + 7) / 8 * 8, c2p = (c2 + 7) / 8 * 8;   // padded: 16-byte aligned GEMM operands
    const int g = OZ_KMAX / c1p < 1 ? 1 : OZ_KMAX / c1p;     // slice pairs per exact FP32 sum
    // the GEMMs of every level (pairs split into runs of at most g) and their levels
    OzLevels lv;
    int ng = 0;
    int p0s[64], nps[64];
    for (int lvl = 2; lvl <= OZ_S + 1; ++lvl)
        for (int p0 = 0; p0 < lvl - 1; p0 += g) {
            lv.lvl[ng] = lvl;
            p0s[ng] = p0;
            nps[ng] = (lvl - 1) - p0 < g ? (lvl - 1) - p0 : g;
            ++ng;
        }
    // row blocks: the FP32 outputs of one block take at most 512 MB
    int64_t nblk = (int64_t)((512ll << 20) / ((int64_t)ng * c2p * 4));
    nblk = nblk / 256 * 256;
    if (nblk < 256) nblk = 256;
    if (nblk > n) nblk = n;
    const size_t bx = align256((size_t)n * OZ_S * c1p * 2);
    const size_t bw = align256((size_t)OZ_S * c1p * c2p * 2);
    const size_t bc = align256((size_t)ng * nblk * c2p * 4);
    const size_t be = align256(sizeof(int) * (n + c2));
    char* buf = nullptr;
    CM_TRY(oz_scratch(ctx, bx + bw + bc + be, &buf));
    __nv_bfloat16* xs = (__nv_bfloat16*)buf;
    __nv_bfloat16* ws = (__nv_bfloat16*)(buf + bx);
    float* Cb = (float*)(buf + bx + bw);
    int* ex = (int*)(buf + bx + bw + bc);
    int* ew = ex + n;
    ProfScope ps(CMSVD_PROF_GEMM, s, 8.0 * ((double)n * c1 + (double)c1 * c2 + (double)n * c2), 2.0 * n * c1 * c2);
    CM_CUDA(cudaMemsetAsync(ew, 0x80, sizeof(int) * c2, s));
    const int grid = ctx->sm_count * 4;
    k_oz_row_exp<<<grid, 256, 0, s>>>(X, ldx, n, c1, ex);
    CM_LAUNCH();
    k_oz_slice_rows<<<ctx->sm_count * 8, 256, 0, s>>>(X, ldx, n, c1, c1p, ex, xs);
    CM_LAUNCH();
    k_oz_col_exp<<<grid, 256, 0, s>>>(W, ldw, c1, c2, ew);
    CM_LAUNCH();
    k_oz_slice_w<<<grid, 256, 0, s>>>(W, ldw, c1, c2, c1p, c2p, ew, ws);
    CM_LAUNCH();
    const float one = 1.f, zero = 0.f;
    for (int64_t r0 = 0; r0 < n; r0 += nblk) {
        const int64_t nr = n - r0 < nblk ? n - r0 : nblk;
        for (int gi = 0; gi < ng; ++gi) {
            const int lvl = lv.lvl[gi], p0 = p0s[gi], np = nps[gi];
            // X slices p0 .. p0+np-1 (rows p0 c1p .. of each column, ld S c1p) against W slices
            // lvl-2-p0 .. lvl-1-p0-np (reversed storage: contiguous, block S-1-q for slice q)
            const __nv_bfloat16* Bm = xs + r0 * (int64_t)OZ_S * c1p + (int64_t)p0 * c1p;
            const int qhi = lvl - 2 - p0;                    // W slice paired with X slice p0
            const __nv_bfloat16* A = ws + (int64_t)(OZ_S - 1 - qhi) * c2p * c1p;
            CM_TRY(blas_ok(cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, c2p, (int)nr, np * c1p, &one, A, CUDA_R_16BF, c2p,
                                        Bm, CUDA_R_16BF, OZ_S * c1p, &zero, Cb + (int64_t)gi * nr * c2p, CUDA_R_32F, c2p,
                                        CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT),
                           "cublasGemmEx (product slices)"));
        }
        k_oz_gemm_epi<<<ctx->sm_count * 8, 256, 0, s>>>(Cb, ng, lv, nr, c2, c2p, ex + r0, ew, Z + r0 * ldz, ldz);
        CM_LAUNCH();
    }
    return CMSVD_OK;
}

// Z (n x c2, ldz) = X (n x c1, ldx) W (c1 x c2, ldw), row-major, in FP64 on cuBLAS's DGEMM: for
// the small square products of the orthogonalization (c x c times c x c), whose 64 x 64 output
// tiles are fewer than the SMs, so the tiled FP64 kernel ran on 16 of 152 SMs; the library
// splits the contraction over the GPU. Deterministic (cuBLAS's GEMMs are run to run).
int gemm_fp64_small(cmsvd_context* ctx, const double* X, int64_t ldx, const double* W, int64_t ldw, double* Z,
                    int64_t ldz, int64_t n, int c1, int c2) {
    cublasHandle_t h;
    CM_TRY(oz_handle(ctx, &h));
    const double one = 1.0, zero = 0.0;
    // column-major view: Z^T (c2 x n) = W^T (c2 x c1) X^T (c1 x n)
    CM_TRY(blas_ok(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, c2, (int)n, c1, &one, W, (int)ldw, X, (int)ldx, &zero, Z,
                               (int)ldz),
                   "cublasDgemm (small product)"));
    return CMSVD_OK;
}

void ozaki_release(cmsvd_context* ctx) {
    if (ctx->blas) cublasDestroy((cublasHandle_t)ctx->blas);
    ctx->blas = nullptr;
    if (ctx->oz_buf) cudaFree(ctx->oz_buf);
    ctx->oz_buf = nullptr;
    ctx->oz_bytes = 0;
}

}  // namespace cmsvd
