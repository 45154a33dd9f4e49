// CSR SpMM, Y = A X with an L-column block: the H X = A^T (A X) product of every shifted
// solve (Alg. 1 / Alg. 2 steps 1-2) and the A V~ product of step 4.
//
// Three operand kinds share one kernel template:
//   F64  FP64 X and Y, FP64 values, FP64 fused multiply-adds;
//   F32  FP32 X and Y, FP32 (or bf16) values, FP32 fused multiply-adds;
//   DF   double-float X and Y (each row: L high parts, then L low parts, FP32), FP32 (or bf16,
//        or split hi + lo FP32) values. Every product a * x_hi is formed exactly (two_prod),
//        the exact errors and the a * x_lo terms are carried in a second FP32 accumulator,
//        and the running sum of the high parts is kept exact with two_sum. The result is
//        accurate to a few units of 2^-48 of sum |a x| while running only on the FP32 pipe,
//        which on GB300 issues 64 times the FMAs of the FP64 pipe.
//
// Layout: a group of LPR lanes owns one row at a time (rows in the matrix's SpMM order) and
// each lane owns VEC consecutive columns, read with one vector load per gathered X row. The
// row's (column, value) pairs are loaded cooperatively and broadcast by shuffles; the X rows of
// U nonzeros are gathered before their multiply-adds, so that U gathers per lane are in flight.
// Each output element is accumulated in the row's storage order by every variant, so results
// are bitwise independent of LPR, U, the column slicing and the grid: the autotuner may pick
// any of them.
#include "internal.cuh"
#include <cstdio>

namespace cmsvd {

// ----------------------------------------------------------------------------- value loaders
struct ValF64 {
    using T = double;
    const double* v;
    __device__ __forceinline__ T load(int64_t p) const { return __ldg(v + p); }
    __device__ __forceinline__ static T zero() { return 0.0; }
    __device__ __forceinline__ static T shfl(unsigned mask, T x, int src, int w) { return __shfl_sync(mask, x, src, w); }
};
struct ValF32 {
    using T = float;
    const float* v;
    __device__ __forceinline__ T load(int64_t p) const { return __ldg(v + p); }
    __device__ __forceinline__ static T zero() { return 0.f; }
    __device__ __forceinline__ static T shfl(unsigned mask, T x, int src, int w) { return __shfl_sync(mask, x, src, w); }
};
struct ValBF16 {   // bf16 bit patterns, widened exactly to FP32
    using T = float;
    const uint16_t* v;
    __device__ __forceinline__ T load(int64_t p) const { return __uint_as_float((uint32_t)__ldg(v + p) << 16); }
    __device__ __forceinline__ static T zero() { return 0.f; }
    __device__ __forceinline__ static T shfl(unsigned mask, T x, int src, int w) { return __shfl_sync(mask, x, src, w); }
};
struct ValSplit {  // a = hi + lo, both FP32 (FP64 values that are not FP32-exact)
    using T = float2;
    const float* hi;
    const float* lo;
    __device__ __forceinline__ T load(int64_t p) const { return make_float2(__ldg(hi + p), __ldg(lo + p)); }
    __device__ __forceinline__ static T zero() { return make_float2(0.f, 0.f); }
    __device__ __forceinline__ static T shfl(unsigned mask, T x, int src, int w) {
        return make_float2(__shfl_sync(mask, x.x, src, w), __shfl_sync(mask, x.y, src, w));
    }
};

// ----------------------------------------------------------------------------- operand policies
template <int VEC> struct VecD;
template <> struct VecD<1> { using T = double; };
template <> struct VecD<2> { using T = double2; };
template <int VEC> struct VecF;
template <> struct VecF<1> { using T = float; };
template <> struct VecF<4> { using T = float4; };

__device__ __forceinline__ double comp(const double& x, int) { return x; }
__device__ __forceinline__ double comp(const double2& x, int q) { return q == 0 ? x.x : x.y; }
__device__ __forceinline__ float comp(const float& x, int) { return x; }
__device__ __forceinline__ float comp(const float4& x, int q) { return q == 0 ? x.x : q == 1 ? x.y : q == 2 ? x.z : x.w; }

template <int VEC_>
struct OpF64 {
    static constexpr int VEC = VEC_;
    using X = typename VecD<VEC>::T;
    struct Acc { double a[VEC]; };
    const double* Xp; int64_t ldx; double* Y; int64_t ldy;
    __device__ __forceinline__ X load(int32_t c, int col) const { return __ldg(reinterpret_cast<const X*>(Xp + (int64_t)c * ldx + col)); }
    __device__ __forceinline__ static X zx() { X x; memset(&x, 0, sizeof(x)); return x; }
    __device__ __forceinline__ static void zero(Acc& a) {
#pragma unroll
        for (int q = 0; q < VEC; ++q) a.a[q] = 0.0;
    }
    __device__ __forceinline__ static void fma(Acc& a, double v, const X& x) {
#pragma unroll
        for (int q = 0; q < VEC; ++q) a.a[q] = __fma_rn(v, comp(x, q), a.a[q]);
    }
    __device__ __forceinline__ void store(const Acc& a, int64_t r, int col) const {
        double* y = Y + r * ldy + col;
#pragma unroll
        for (int q = 0; q < VEC; ++q) y[q] = a.a[q];
    }
};

template <int VEC_>
struct OpF32 {
    static constexpr int VEC = VEC_;
    using X = typename VecF<VEC>::T;
    struct Acc { float a[VEC]; };
    const float* Xp; int64_t ldx; float* Y; int64_t ldy;
    __device__ __forceinline__ X load(int32_t c, int col) const { return __ldg(reinterpret_cast<const X*>(Xp + (int64_t)c * ldx + col)); }
    __device__ __forceinline__ static X zx() { X x; memset(&x, 0, sizeof(x)); return x; }
    __device__ __forceinline__ static void zero(Acc& a) {
#pragma unroll
        for (int q = 0; q < VEC; ++q) a.a[q] = 0.f;
    }
    __device__ __forceinline__ static void fma(Acc& a, float v, const X& x) {
#pragma unroll
        for (int q = 0; q < VEC; ++q) a.a[q] = __fmaf_rn(v, comp(x, q), a.a[q]);
    }
    __device__ __forceinline__ void store(const Acc& a, int64_t r, int col) const {
        float* y = Y + r * ldy + col;
#pragma unroll
        for (int q = 0; q < VEC; ++q) y[q] = a.a[q];
    }
};

// one compensated multiply-add: (h, l) += a * (xh + xl), a a single FP32 value
__device__ __forceinline__ void df_madd(float& h, float& l, float a, float xh, float xl) {
    float p, e, s, t;
    two_prod(a, xh, p, e);
    const float c = __fmaf_rn(a, xl, e);
    two_sum(h, p, s, t);
    h = s;
    l = __fadd_rn(l, __fadd_rn(t, c));
}
// the same with a = ah + al
__device__ __forceinline__ void df_madd(float& h, float& l, float2 a, float xh, float xl) {
    float p, e, s, t;
    two_prod(a.x, xh, p, e);
    const float c = __fmaf_rn(a.y, xh, __fmaf_rn(a.x, xl, e));
    two_sum(h, p, s, t);
    h = s;
    l = __fadd_rn(l, __fadd_rn(t, c));
}

template <int VEC_>
struct OpDF {
    static constexpr int VEC = VEC_;
    using V = typename VecF<VEC>::T;
    struct X { V h, l; };
    struct Acc { float h[VEC], l[VEC]; };
    const float* Xp; int64_t ldx; float* Y; int64_t ldy; int L;
    __device__ __forceinline__ X load(int32_t c, int col) const {
        const float* x = Xp + (int64_t)c * ldx + col;
        X r;
        r.h = __ldg(reinterpret_cast<const V*>(x));
        r.l = __ldg(reinterpret_cast<const V*>(x + L));
        return r;
    }
    __device__ __forceinline__ static X zx() { X x; memset(&x, 0, sizeof(x)); return x; }
    __device__ __forceinline__ static void zero(Acc& a) {
#pragma unroll
        for (int q = 0; q < VEC; ++q) { a.h[q] = 0.f; a.l[q] = 0.f; }
    }
    template <typename VT>
    __device__ __forceinline__ static void fma(Acc& a, VT v, const X& x) {
#pragma unroll
        for (int q = 0; q < VEC; ++q) df_madd(a.h[q], a.l[q], v, comp(x.h, q), comp(x.l, q));
    }
    __device__ __forceinline__ void store(const Acc& a, int64_t r, int col) const {
        float* y = Y + r * ldy + col;
#pragma unroll
        for (int q = 0; q < VEC; ++q) {   // two_sum: the low part may exceed the high part after cancellation
            float h, l;
            two_sum(a.h[q], a.l[q], h, l);
            y[q] = h;
            y[L + q] = l;
        }
    }
};

// ----------------------------------------------------------------------------- the kernel
// The X rows of up to U nonzeros of one chunk (LPR consecutive nonzeros of a row, one pair per
// lane) are gathered, then multiplied in storage order.
template <class Op, class Val, int LPR, int U>
__device__ __forceinline__ void spmm_chunk(const Op& op, unsigned mask, int32_t mc, typename Val::T mv, int cnt,
                                           int col, bool on, typename Op::Acc& acc) {
    int k0 = 0;
    for (; k0 + U <= cnt; k0 += U) {
        typename Op::X xv[U];
        typename Val::T vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t c = __shfl_sync(mask, mc, k0 + u, LPR);
            vv[u] = Val::shfl(mask, mv, k0 + u, LPR);
            xv[u] = on ? op.load(c, col) : Op::zx();
        }
#pragma unroll
        for (int u = 0; u < U; ++u) Op::fma(acc, vv[u], xv[u]);
    }
    for (; k0 < cnt; ++k0) {
        const int32_t c = __shfl_sync(mask, mc, k0, LPR);
        const typename Val::T v = Val::shfl(mask, mv, k0, LPR);
        if (on) Op::fma(acc, v, op.load(c, col));
    }
}

// Rows are taken in a software pipeline two rows deep: while a group multiplies row k, the
// (column, value) pairs of its row k+1 (its first 2 LPR nonzeros) and the row pointers of row
// k+2 are already in flight, so the only latency left on a row's path is its X gathers.
template <class Op, class Val, int LPR, int U>
__global__ void __launch_bounds__(256) k_spmm_vec(Op op, Val val, const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ colidx, int64_t rows, int c_lo, int c_hi,
                                                  const int32_t* __restrict__ order) {
    using VT = typename Val::T;
    constexpr int VEC = Op::VEC;
    const int lane = threadIdx.x % LPR;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / LPR;
    const unsigned mask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << ((threadIdx.x & 31) / LPR * LPR));
    auto row_of = [&](int64_t rr) -> int64_t { return order ? (int64_t)__ldg(order + rr) : rr; };
    // pipeline state: row k (cur) with its pairs, row k+1 (nxt) with its pairs, row k+2 (far) pointers
    int64_t rr = group;
    if (rr >= rows) return;
    int64_t r = row_of(rr), s = __ldg(rowptr + r), e = __ldg(rowptr + r + 1);
    int64_t rn = 0, sn = 0, en = 0;
    const bool has1 = rr + ngroups < rows;
    if (has1) { rn = row_of(rr + ngroups); sn = __ldg(rowptr + rn); en = __ldg(rowptr + rn + 1); }
    int32_t c0a = 0, c1a = 0;
    VT v0a = Val::zero(), v1a = Val::zero();
    if (s + lane < e) { c0a = __ldg(colidx + s + lane); v0a = val.load(s + lane); }
    if (s + LPR + lane < e) { c1a = __ldg(colidx + s + LPR + lane); v1a = val.load(s + LPR + lane); }
    for (;;) {
        const bool has_n = rr + ngroups < rows;
        const bool has_f = rr + 2 * ngroups < rows;
        // issue: pairs of row k+1, pointers of row k+2
        int32_t c0b = 0, c1b = 0;
        VT v0b = Val::zero(), v1b = Val::zero();
        if (has_n) {
            if (sn + lane < en) { c0b = __ldg(colidx + sn + lane); v0b = val.load(sn + lane); }
            if (sn + LPR + lane < en) { c1b = __ldg(colidx + sn + LPR + lane); v1b = val.load(sn + LPR + lane); }
        }
        int64_t rf = 0, sf = 0, ef = 0;
        if (has_f) { rf = row_of(rr + 2 * ngroups); sf = __ldg(rowptr + rf); ef = __ldg(rowptr + rf + 1); }
        // row k
        for (int cb = c_lo; cb < c_hi; cb += LPR * VEC) {
            const int col = cb + lane * VEC;
            const bool on = col < c_hi;
            typename Op::Acc acc;
            Op::zero(acc);
            const int64_t len = e - s;
            spmm_chunk<Op, Val, LPR, U>(op, mask, c0a, v0a, (int)(len < LPR ? len : LPR), col, on, acc);
            if (len > LPR)
                spmm_chunk<Op, Val, LPR, U>(op, mask, c1a, v1a, (int)(len - LPR < LPR ? len - LPR : LPR), col, on, acc);
            for (int64_t p0 = s + 2 * LPR; p0 < e; p0 += LPR) {   // rows longer than 2 LPR
                const int64_t p = p0 + lane;
                int32_t mc = 0;
                VT mv = Val::zero();
                if (p < e) { mc = __ldg(colidx + p); mv = val.load(p); }
                spmm_chunk<Op, Val, LPR, U>(op, mask, mc, mv, (int)((e - p0) < LPR ? (e - p0) : LPR), col, on, acc);
            }
            if (on) op.store(acc, r, col);
        }
        if (!has_n) break;
        rr += ngroups;
        r = rn; s = sn; e = en;
        c0a = c0b; v0a = v0b; c1a = c1b; v1a = v1b;
        rn = rf; sn = sf; en = ef;
    }
}

// Long rows (a few rows holding most nonzeros, e.g. the transpose of a matrix whose columns are
// image pixels): one CTA per row. Its 256 / LPR groups take contiguous, equal slices of the row,
// and their partial sums are added in slice order, so the result is deterministic (the summation
// order differs from k_spmm_vec's). FP64 and FP32 operands only.
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
                for (int k = 0; k < cnt; ++k) {
                    const int32_t col = __shfl_sync(mask, mc, k, LPR);
                    const T v = __shfl_sync(mask, mv, k, LPR);
                    const T* xr = X + (int64_t)col * ldx + c0 + lane;
#pragma unroll
                    for (int q = 0; q < CPL; ++q)
                        if (c0 + lane + q * LPR < L) acc[q] = fma(v, __ldg(xr + q * LPR), acc[q]);
                }
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

// ----------------------------------------------------------------------------- launch plumbing
// Candidate (lanes per row, gathers in flight) pairs; the kernel template is instantiated for
// each. The column slicing and the grid are run-time choices.
struct Variant { int lpr, unroll; };
static const Variant kVariants[] = {{1, 4}, {1, 8}, {2, 4}, {2, 8}, {4, 4}, {4, 8}, {8, 4}, {8, 8},
                                    {16, 4}, {16, 8}, {32, 4}, {32, 8}};

template <class Op, class Val>
static const void* kernel_ptr(int lpr, int unroll) {
#define CM_K(LP, UU) if (lpr == LP && unroll == UU) return (const void*)k_spmm_vec<Op, Val, LP, UU>;
    CM_K(1, 4) CM_K(1, 8) CM_K(2, 4) CM_K(2, 8) CM_K(4, 4) CM_K(4, 8) CM_K(8, 4) CM_K(8, 8)
    CM_K(16, 4) CM_K(16, 8) CM_K(32, 4) CM_K(32, 8)
#undef CM_K
    return nullptr;
}

template <class Op, class Val>
static int launch_vec(const Csr& A, const Op& op, const Val& val, int L, const SpmmCfg& cfg, cudaStream_t s) {
    const void* fn = kernel_ptr<Op, Val>(cfg.lpr, cfg.unroll);
    if (!fn) { set_error("no SpMM variant with %d lanes x %d gathers", cfg.lpr, cfg.unroll); return CMSVD_INVALID_ARG; }
    int per_sm = cfg.blocks_per_sm;
    if (per_sm <= 0) {
        per_sm = 1;
        CM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0));
        if (per_sm < 1) per_sm = 1;
    }
    const int64_t rows_per_block = 256 / cfg.lpr;
    int64_t grid = (A.m + rows_per_block - 1) / rows_per_block;
    const int64_t cap = (int64_t)per_sm * (A.sm_count > 0 ? A.sm_count : 1);
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    const int slices = cfg.slices < 1 ? 1 : cfg.slices;
    const int step = ((L / slices + Op::VEC - 1) / Op::VEC) * Op::VEC;
    for (int c_lo = 0; c_lo < L; c_lo += step) {
        int c_hi = c_lo + step < L ? c_lo + step : L;
        Op o = op;
        Val v = val;
        const int64_t* rp = A.rowptr;
        const int32_t* ci = A.colidx;
        int64_t rows = A.m;
        const int32_t* ord = cfg.natural ? nullptr : A.row_order;
        void* args[] = {&o, &v, &rp, &ci, &rows, &c_lo, &c_hi, &ord};
        CM_CUDA(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(256), args, 0, s));
        note_launch();
    }
    return CMSVD_OK;
}

static SpmmCfg default_cfg(int vec, int L) {
    SpmmCfg c;
    int lpr = 4;
    while (lpr < 32 && lpr * vec < L) lpr *= 2;
    c.lpr = lpr;
    c.unroll = 8;
    c.slices = 1;
    return c;
}

// callers hold A.tune->mu
static SpmmTuneEntry* tune_find(Csr& A, int kind, int L) {
    for (auto& t : A.tune->e)
        if (t.kind == kind && t.L == L) return &t;
    return nullptr;
}

static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) { cudaGetLastError(); return true; }
    return cs != cudaStreamCaptureStatusNone;
}

// Times every candidate on the call's own buffers (the product is pure, so the last launch
// leaves the right result) and keeps the fastest for (A, kind, L).
template <class Op, class Val>
static int autotune(Csr& A, int kind, int L, const Op& op, const Val& val, cudaStream_t s, SpmmCfg* best_out) {
    cudaEvent_t e0, e1;
    CM_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(cudaGetLastError(), "event", __FILE__, __LINE__); }
    SpmmCfg best = default_cfg(Op::VEC, L);
    float best_ms = 1e30f;
    int st = CMSVD_OK;
    // Column slices (each launch covers L / slices columns for all rows, so that the gathered
    // part of X can stay in L2) with lanes per row matched to the slice width: one to four
    // passes of LPR * VEC columns per slice.
    const int nvec = (L + Op::VEC - 1) / Op::VEC;
    for (int nat = 0; nat < (A.row_order ? 2 : 1) && st == CMSVD_OK; ++nat)
    for (int sl = 1; sl <= 8 && sl <= nvec && st == CMSVD_OK; sl *= 2)
    for (const Variant& v : kVariants) {
        const int w = ((L / sl + Op::VEC - 1) / Op::VEC) * Op::VEC;      // columns per slice
        if (v.lpr * Op::VEC > w && v.lpr > 1) continue;                 // idle lanes
        if (v.lpr * Op::VEC * 4 < w) continue;                          // more than four passes per row
        {
            SpmmCfg c;
            c.lpr = v.lpr;
            c.unroll = v.unroll;
            c.slices = sl;
            c.natural = nat;
            st = launch_vec(A, op, val, L, c, s);                      // warm
            if (st != CMSVD_OK) break;
            float ms = 0.f;
            cudaError_t ce = cudaEventRecord(e0, s);
            for (int rep = 0; rep < 2 && st == CMSVD_OK; ++rep) st = launch_vec(A, op, val, L, c, s);
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce != cudaSuccess) st = cuda_fail(ce, "SpMM autotune timing", __FILE__, __LINE__);
            if (st != CMSVD_OK) break;
            if (ms < best_ms) { best_ms = ms; best = c; best.ms = ms / 2; }
        }
        if (st != CMSVD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CMSVD_OK) return st;
    SpmmTuneEntry* slot = &A.tune->e[63];                              // a full cache reuses its last entry
    for (auto& t : A.tune->e)
        if (t.kind < 0) { slot = &t; break; }
    slot->kind = kind;
    slot->L = L;
    slot->cfg = best;
    *best_out = best;
    // leave the result of the chosen configuration in Y
    return launch_vec(A, op, val, L, best, s);
}

// Tuning runs only inside spmm_tune (the Krylov solver before its graph capture, and the
// public SpMM entry points); other products (the Rayleigh-Ritz steps, whose widths change
// from solve to solve) take a cached pick or the default configuration.
static thread_local bool t_allow_tune = false;

template <class Op, class Val>
static int run_vec(Csr& A, int kind, int L, const Op& op, const Val& val, cudaStream_t s) {
    // small products are launch-bound: not tuned
    if (A.nnz * (int64_t)L < (int64_t)1 << 24) return launch_vec(A, op, val, L, default_cfg(Op::VEC, L), s);
    std::unique_lock<std::mutex> lk(A.tune->mu, std::try_to_lock);
    if (!lk.owns_lock()) return launch_vec(A, op, val, L, default_cfg(Op::VEC, L), s);   // another stream is tuning
    SpmmTuneEntry* t = tune_find(A, kind, L);
    if (t) {
        const SpmmCfg c = t->cfg;
        lk.unlock();
        return launch_vec(A, op, val, L, c, s);
    }
    if (!t_allow_tune || capturing(s)) return launch_vec(A, op, val, L, default_cfg(Op::VEC, L), s);
    SpmmCfg c;
    return autotune(A, kind, L, op, val, s, &c);
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// tuning keys: kind * 8 + vector flag (different kernels for aligned and scalar operands)
static int key(int kind, int vec) { return kind * 8 + (vec > 1 ? 1 : 0); }

// ----------------------------------------------------------------------------- FP64
int spmm(const Csr& Ac, int L, const double* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t s) {
    Csr& A = const_cast<Csr&>(Ac);
    if (A.m == 0 || L <= 0) return CMSVD_OK;
    const double e = 8.0;
    ProfScope ps(CMSVD_PROF_SPMM, s, (e + 4.0) * A.nnz + 8.0 * (A.m + 1) + e * L * (A.n + A.m), 2.0 * A.nnz * L);
    if (A.max_row > 2048) {
        const int sms = A.sm_count > 0 ? A.sm_count : 1;
        const unsigned grid = (unsigned)(A.m < sms * 8 ? A.m : sms * 8);
        if (L <= 8) k_spmm_rowcta<double, 8, 1><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, A.vals, A.m, L, X, ldx, Y, ldy, A.row_order);
        else if (L <= 16) k_spmm_rowcta<double, 16, 1><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, A.vals, A.m, L, X, ldx, Y, ldy, A.row_order);
        else if (L <= 32) k_spmm_rowcta<double, 32, 1><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, A.vals, A.m, L, X, ldx, Y, ldy, A.row_order);
        else k_spmm_rowcta<double, 32, 4><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, A.vals, A.m, L, X, ldx, Y, ldy, A.row_order);
        CM_LAUNCH();
        return CMSVD_OK;
    }
    ValF64 val{A.vals};
    if (L % 2 == 0 && ldx % 2 == 0 && ldy % 2 == 0 && aligned16(X) && aligned16(Y))
        return run_vec(A, key(SPMM_KIND_F64, 2), L, OpF64<2>{X, ldx, Y, ldy}, val, s);
    return run_vec(A, key(SPMM_KIND_F64, 1), L, OpF64<1>{X, ldx, Y, ldy}, val, s);
}

// ----------------------------------------------------------------------------- FP32
int spmm(const Csr& Ac, int L, const float* X, int64_t ldx, float* Y, int64_t ldy, cudaStream_t s) {
    Csr& A = const_cast<Csr&>(Ac);
    if (!A.vals_f) { set_error("FP32 values of A were not made"); return CMSVD_INVALID_ARG; }
    if (A.m == 0 || L <= 0) return CMSVD_OK;
    const double ev = A.storage == CMSVD_STORE_BF16 ? 2.0 : 4.0;
    ProfScope ps(CMSVD_PROF_SPMM, s, (ev + 4.0) * A.nnz + 8.0 * (A.m + 1) + 4.0 * L * (A.n + A.m), 2.0 * A.nnz * L);
    if (A.max_row > 2048) {
        const int sms = A.sm_count > 0 ? A.sm_count : 1;
        const unsigned grid = (unsigned)(A.m < sms * 8 ? A.m : sms * 8);
        if (L <= 8) k_spmm_rowcta<float, 8, 1><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, A.vals_f, A.m, L, X, ldx, Y, ldy, A.row_order);
        else if (L <= 16) k_spmm_rowcta<float, 16, 1><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, A.vals_f, A.m, L, X, ldx, Y, ldy, A.row_order);
        else if (L <= 32) k_spmm_rowcta<float, 32, 1><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, A.vals_f, A.m, L, X, ldx, Y, ldy, A.row_order);
        else k_spmm_rowcta<float, 32, 4><<<grid, 256, 0, s>>>(A.rowptr, A.colidx, A.vals_f, A.m, L, X, ldx, Y, ldy, A.row_order);
        CM_LAUNCH();
        return CMSVD_OK;
    }
    const bool vec = L % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 && aligned16(X) && aligned16(Y);
    if (A.storage == CMSVD_STORE_BF16 && A.vals_h) {
        if (vec) return run_vec(A, key(SPMM_KIND_F32, 4) + 2, L, OpF32<4>{X, ldx, Y, ldy}, ValBF16{A.vals_h}, s);
        return run_vec(A, key(SPMM_KIND_F32, 1) + 2, L, OpF32<1>{X, ldx, Y, ldy}, ValBF16{A.vals_h}, s);
    }
    if (vec) return run_vec(A, key(SPMM_KIND_F32, 4), L, OpF32<4>{X, ldx, Y, ldy}, ValF32{A.vals_f}, s);
    return run_vec(A, key(SPMM_KIND_F32, 1), L, OpF32<1>{X, ldx, Y, ldy}, ValF32{A.vals_f}, s);
}

// ----------------------------------------------------------------------------- double-float
int spmm_df(const Csr& Ac, int L, const float* X, int64_t ldx, float* Y, int64_t ldy, cudaStream_t s) {
    Csr& A = const_cast<Csr&>(Ac);
    if (!A.vals_f) { set_error("FP32 values of A were not made"); return CMSVD_INVALID_ARG; }
    if (A.m == 0 || L <= 0) return CMSVD_OK;
    const bool split = A.f32_exact == 0;
    const double ev = split ? 8.0 : (A.storage == CMSVD_STORE_BF16 ? 2.0 : 4.0);
    // flops: the FP32 operations of the compensated multiply-add (11, or 12 with split values)
    ProfScope ps(CMSVD_PROF_SPMM, s, (ev + 4.0) * A.nnz + 8.0 * (A.m + 1) + 8.0 * L * (A.n + A.m),
                 (split ? 12.0 : 11.0) * A.nnz * L);
    const bool vec = L % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 && aligned16(X) && aligned16(Y);
    const int kv = vec ? 4 : 1;
    if (split) {
        ValSplit v{A.vals_f, A.vals_lo};
        if (vec) return run_vec(A, key(SPMM_KIND_DF, kv) + 4, L, OpDF<4>{X, ldx, Y, ldy, L}, v, s);
        return run_vec(A, key(SPMM_KIND_DF, kv) + 4, L, OpDF<1>{X, ldx, Y, ldy, L}, v, s);
    }
    if (A.storage == CMSVD_STORE_BF16 && A.vals_h) {
        ValBF16 v{A.vals_h};
        if (vec) return run_vec(A, key(SPMM_KIND_DF, kv) + 2, L, OpDF<4>{X, ldx, Y, ldy, L}, v, s);
        return run_vec(A, key(SPMM_KIND_DF, kv) + 2, L, OpDF<1>{X, ldx, Y, ldy, L}, v, s);
    }
    ValF32 v{A.vals_f};
    if (vec) return run_vec(A, key(SPMM_KIND_DF, kv), L, OpDF<4>{X, ldx, Y, ldy, L}, v, s);
    return run_vec(A, key(SPMM_KIND_DF, kv), L, OpDF<1>{X, ldx, Y, ldy, L}, v, s);
}

// The autotuner's pick for (A, kind, L), if it has run: vectorized operands first.
bool spmm_tuned(const Csr& A, int kind, int L, SpmmCfg* cfg) {
    std::lock_guard<std::mutex> lk(A.tune->mu);
    const SpmmTuneEntry* found = nullptr;
    for (const auto& t : A.tune->e) {
        if (t.kind >= kind * 8 && t.kind < kind * 8 + 8 && t.L == L) {
            if (!found || ((t.kind & 1) && !(found->kind & 1))) found = &t;
        }
    }
    if (!found) return false;
    *cfg = found->cfg;
    return true;
}

// Runs the autotuner (if it has not run) on the given buffers: one product is computed.
int spmm_tune(Csr& A, int kind, int L, const void* X, int64_t ldx, void* Y, int64_t ldy, cudaStream_t s) {
    t_allow_tune = true;
    int st;
    if (kind == SPMM_KIND_F64) st = spmm(A, L, (const double*)X, ldx, (double*)Y, ldy, s);
    else if (kind == SPMM_KIND_F32) st = spmm(A, L, (const float*)X, ldx, (float*)Y, ldy, s);
    else st = spmm_df(A, L, (const float*)X, ldx, (float*)Y, ldy, s);
    t_allow_tune = false;
    return st;
}

}  // namespace cmsvd
