// Internal declarations shared by the CUDA translation units of libcmsvd.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <memory>
#include <mutex>
#include "cmsvd.h"

namespace cmsvd {

// ----------------------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CM_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e__ = (call);                                                  \
        if (e__ != cudaSuccess) return ::cmsvd::cuda_fail(e__, #call, __FILE__, __LINE__); \
    } while (0)
#define CM_LAUNCH()               \
    do {                          \
        ::cmsvd::note_launch();   \
        CM_CUDA(cudaGetLastError()); \
    } while (0)
#define CM_TRY(expr)                                                               \
    do {                                                                           \
        int s__ = (expr);                                                          \
        if (s__ != CMSVD_OK) return s__;                                           \
    } while (0)

// ----------------------------------------------------------------------------- launch counting / profiling
// One profiler per host thread, active for the duration of one library call.
// Launch counting is always on; event timing only when params.profile is set.
struct Profiler {
    bool timing = false;
    int capture_depth = 0;        // > 0 while a CUDA graph is being captured
    int64_t launches = 0;         // kernels launched (graph nodes added per graph launch)
    int64_t captured = 0;         // kernels recorded into the graph being captured
    struct Rec { int cls; cudaEvent_t e0, e1; double bytes, flops; int64_t launches; };
    Rec recs[4096];
    int nrec = 0;
};
Profiler& prof();
inline void note_launch() {
    Profiler& p = prof();
    if (p.capture_depth > 0) ++p.captured; else ++p.launches;
}
// Times the launches issued inside its scope on stream s as one record of class cls.
struct ProfScope {
    int idx = -1;
    cudaStream_t stream_ = nullptr;
    ProfScope(int cls, cudaStream_t s, double bytes, double flops, int64_t launches = 1);
    ~ProfScope();
};
void prof_reset(bool timing);
void prof_collect(cmsvd_stats* st);   // synchronizes the recorded events

// ----------------------------------------------------------------------------- objects
// SpMM configuration picked by the autotuner (spmm.cu) for one (operand kind, L) pair.
// natural = 1 takes the rows in storage order instead of the locality order (row_order).
struct SpmmCfg { int lpr = 0, unroll = 0, slices = 1, blocks_per_sm = 0, natural = 0; float ms = 0.f; };
struct SpmmTuneEntry { int kind = -1, L = 0; SpmmCfg cfg; };
// Autotuner cache of one stored matrix, shared by its shallow per-stream views (serving):
// one thread tunes at a time; the others use the default configuration meanwhile.
struct SpmmTuneCache {
    std::mutex mu;
    SpmmTuneEntry e[64];
};

struct Csr {
    int64_t m = 0, n = 0, nnz = 0;
    int64_t* rowptr = nullptr;   // device, m+1
    int32_t* colidx = nullptr;   // device, nnz
    double* vals = nullptr;      // device, nnz: the values as FP64 (after rounding to the storage precision)
    float* vals_f = nullptr;     // device, nnz: FP32 values (made on demand for FP32 / double-float products)
    float* vals_lo = nullptr;    // device, nnz: a - fl32(a), made with vals_f when some value is not FP32-exact
    uint16_t* vals_h = nullptr;  // device, nnz: bf16 bit patterns (storage BF16)
    int storage = CMSVD_STORE_FP64;
    int f32_exact = -1;          // 1: every value is FP32-representable (known once vals_f exists)
    int sm_count = 0;
    int64_t max_row = 0;         // longest row (nonzeros); long rows switch the SpMM to one CTA per row
    int32_t* row_order = nullptr; // device, m: rows sorted by their first column (SpMM processing order)
    std::shared_ptr<SpmmTuneCache> tune = std::make_shared<SpmmTuneCache>();   // autotuner cache (host)
};

struct Components {             // connected components of the column graph (A^T A)
    bool ready = false;
    int64_t count = 0;
    int64_t max_size = 0;
    // columns grouped by component, components grouped by size (device)
    int64_t n_groups = 0;
    int32_t* group_size = nullptr;      // host copy [n_groups]
    int64_t* group_count = nullptr;     // host [n_groups]
    int64_t* group_col_off = nullptr;   // host [n_groups] offset into cols[]
    int32_t* cols = nullptr;            // device [n], columns ordered by (group, component, local)
    int64_t* comp_row_ptr = nullptr;    // device [count+1], rows of each component (CSR rows of A)
    int32_t* comp_rows = nullptr;       // device [rows with entries]
    int64_t* comp_first = nullptr;      // host [count+1] first column slot of each component in cols[]
    int64_t* comp_first_dev = nullptr;  // device copy
    int32_t* col_local = nullptr;       // device [n], local index of a column inside its component
};

// ----------------------------------------------------------------------------- double-float arithmetic
// A value x is carried as an unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2
// after normalization). Building blocks, all with explicit round-to-nearest intrinsics so that
// the compiler neither contracts nor reorders them:
//   two_sum       Knuth's TwoSum: s + e == a + b exactly, for any a, b;
//   fast_two_sum  Dekker's Fast2Sum: the same when |a| >= |b| (or a == 0);
//   two_prod      the FMA-based exact product: p + e == a * b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

}  // namespace cmsvd

struct cmsvd_context {
    int device = 0;
    cudaStream_t user = nullptr;       // borrowed
    cudaStream_t s = nullptr;          // owned, non-blocking: all library work runs here
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int sm_count = 0;
    int* pinned = nullptr;             // host-pinned flags for polling
    int dense_arith = 0;               // 0: FP64-accurate tall products on BF16 tensor cores (ozaki.cu); 1: FP64 pipe
    void* blas = nullptr;              // cuBLAS handle of the tensor-core slice products (made on first use)
    void* oz_buf = nullptr;            // their scratch, kept between calls
    size_t oz_bytes = 0;
};

struct cmsvd_matrix {
    cmsvd_context* ctx = nullptr;
    cmsvd::Csr A, At;
    double norm_est = 0.0;             // cached ||A||_2 estimate (0 = not yet)
    double ms_components = 0.0;        // host time of the components build (0 = not built)
    cmsvd::Components comp;
};

struct cmsvd_result {
    int64_t m = 0, n = 0, t = 0;
    cmsvd_context* ctx = nullptr;
    double* sigma = nullptr;   // device pointers into the caller workspace
    double* U = nullptr;       // m x t column-major
    double* V = nullptr;       // n x t column-major
    double* res_u = nullptr;
    double* res_v = nullptr;
    double* tau = nullptr;
    double* res_est = nullptr; // null unless the solve ran with estimate = 1
    cmsvd_stats stats{};
};

namespace cmsvd {

// The context of the entry point running on this host thread (set by Session::open).
cmsvd_context*& current_ctx();

// FP64-accurate tall-skinny products from exact BF16 tensor-core slice products (ozaki.cu).
bool ozaki_applies(const cmsvd_context* ctx, int64_t n, int c1, int c2);
int gram_ozaki(cmsvd_context* ctx, const double* X, int64_t ldx, int c1, const double* Y, int64_t ldy, int c2,
               int64_t n, double* G, int64_t ldg);
int gemm_ozaki(cmsvd_context* ctx, const double* X, int64_t ldx, const double* W, int64_t ldw, double* Z, int64_t ldz,
               int64_t n, int c1, int c2);
int gemm_fp64_small(cmsvd_context* ctx, const double* X, int64_t ldx, const double* W, int64_t ldw, double* Z,
                    int64_t ldz, int64_t n, int c1, int c2);
void ozaki_release(cmsvd_context* ctx);

// ----------------------------------------------------------------------------- entry-point session
// An entry point's work runs on the context's internal stream: open() makes the context's
// device current (remembering the caller's), orders the internal stream after the caller's
// stream, and close() orders the caller's stream after the internal one and makes the caller's
// device current again. The destructor does the same on an early error return, so that what
// the caller queues next (freeing its buffers, say) waits for the kernels already queued, and
// the caller's current device is never left changed.
struct Session {
    cmsvd_context* c = nullptr;
    int prev = -1;
    cmsvd_context* outer = nullptr;
    Session() = default;
    Session(const Session&) = delete;
    Session& operator=(const Session&) = delete;
    ~Session() {
        if (c) {
            cudaEventRecord(c->ev_out, c->s);
            cudaStreamWaitEvent(c->user, c->ev_out, 0);
        }
        restore();
    }
    void restore() {
        if (prev >= 0) {
            cudaSetDevice(prev);
            current_ctx() = outer;
        }
        prev = -1;
    }
    int open(cmsvd_context* ctx) {
        int d = -1;
        CM_CUDA(cudaGetDevice(&d));
        prev = d;
        outer = current_ctx();
        current_ctx() = ctx;
        CM_CUDA(cudaSetDevice(ctx->device));
        CM_CUDA(cudaEventRecord(ctx->ev_in, ctx->user));
        CM_CUDA(cudaStreamWaitEvent(ctx->s, ctx->ev_in, 0));
        c = ctx;
        return CMSVD_OK;
    }
    int close() {
        cmsvd_context* x = c;
        c = nullptr;
        cudaError_t e = cudaEventRecord(x->ev_out, x->s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(x->user, x->ev_out, 0);
        restore();
        if (e != cudaSuccess) return cuda_fail(e, "rejoin the caller's stream", __FILE__, __LINE__);
        return CMSVD_OK;
    }
};

// ----------------------------------------------------------------------------- workspace arena
// Bump allocator over the caller's workspace. With base == nullptr it only
// measures, so the size query and the solve run the same allocation sequence.
struct Arena {
    char* base = nullptr;
    size_t off = 0, cap = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    bool fits() const { return base == nullptr || off <= cap; }
};

// ----------------------------------------------------------------------------- launchers (csr.cu)
int csr_upload_validate(cmsvd_context* ctx, int64_t m, int64_t n, int64_t nnz, const int64_t* rowptr,
                        const int32_t* colidx, const double* vals, int where, Csr* out);
int csr_transpose(cmsvd_context* ctx, const Csr& A, Csr* At);
// Rounds A's values to the storage precision (cmsvd_storage) in place; bf16 also keeps the
// 16-bit patterns. CMSVD_INVALID_MATRIX when a value overflows the storage precision.
int csr_round_storage(cmsvd_context* ctx, Csr* A, int storage);
void csr_free(Csr* A);
// Y (rows x L, ldy) = A X (X: ncols x L, ldx); every kernel variant sums each output
// element in the row's storage order, so the result does not depend on the variant.
int spmm(const Csr& A, int L, const double* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t s);
// FP32 SpMM: FP32 values of A (A.vals_f, or the bf16 values for bf16 storage), FP32 accumulation.
int spmm(const Csr& A, int L, const float* X, int64_t ldx, float* Y, int64_t ldy, cudaStream_t s);
// Double-float SpMM (FP32 arithmetic, error-free products and compensated sums): X and Y
// hold each row as L high parts followed by L low parts (ld in floats, >= 2 L).
int spmm_df(const Csr& A, int L, const float* X, int64_t ldx, float* Y, int64_t ldy, cudaStream_t s);
// Runs the autotuner for (A, kind, L) now, on the given buffers, outside any stream capture.
enum { SPMM_KIND_F64 = 0, SPMM_KIND_F32 = 1, SPMM_KIND_DF = 2 };
int spmm_tune(Csr& A, int kind, int L, const void* X, int64_t ldx, void* Y, int64_t ldy, cudaStream_t s);
bool spmm_tuned(const Csr& A, int kind, int L, SpmmCfg* cfg);
int csr_make_fp32(cmsvd_matrix* M);   // vals_f (and vals_lo when needed) of A and A^T
int components_build(cmsvd_matrix* M);
void components_free(Components* c);

// ----------------------------------------------------------------------------- quadrature (krylov.cu)
struct QuadParams { double a, b, alpha; int N, variant; };
// quad: device array of 3*J double2 = (shift, weight, scaled) per point j.
int quadrature_device(const QuadParams& q, double2* quad, cudaStream_t s);

// ----------------------------------------------------------------------------- filter solves
// S (n x L(M+1), ld = L(M+1)) = 2 Re sum_j w_j scaled_j^k (s_j I - A^T A)^{-1} X  for k = 0..Mk-1
struct SolveOut {
    int64_t iters = 0;
    int converged = 1;
    int breakdown = 0;
    int refine_rounds = 0;
    double refine_residual = 0.0;
};
size_t krylov_workspace(const cmsvd_matrix* A, const cmsvd_params* p);
int krylov_moments(cmsvd_matrix* A, const cmsvd_params* p, const double2* quad, int Mk,
                   const double* X, int64_t ldx, double* S, int64_t lds, Arena& ws, SolveOut* out);
size_t direct_workspace(const cmsvd_matrix* A, const cmsvd_params* p);
int direct_moments(cmsvd_matrix* A, const cmsvd_params* p, const double2* quad, int Mk,
                   const double* X, int64_t ldx, double* S, int64_t lds, Arena& ws);
size_t dense_workspace(const cmsvd_matrix* A, const cmsvd_params* p);
int dense_moments(cmsvd_matrix* A, const cmsvd_params* p, const double2* quad, int Mk,
                  const double* X, int64_t ldx, double* S, int64_t lds, Arena& ws);
int norm_estimate(cmsvd_matrix* A, Arena& ws, double* norm_out);

// Persistent outputs of one solve (capacity L M each; U m x c, V n x c).
struct RitzOut { double *sigma, *U, *V, *res_u, *res_v, *tau, *res_est; };

// ----------------------------------------------------------------------------- dense (dense.cu)
// G (c1 x c2, row-major) = X^T Y, X: n x c1 (ldx), Y: n x c2 (ldy). Deterministic.
int gram(const double* X, int64_t ldx, int c1, const double* Y, int64_t ldy, int c2, int64_t n,
         double* G, double* partials, size_t partials_cap, int sm_count, cudaStream_t s);
size_t gram_partials_size(int c1, int c2, int64_t n, int sm_count, int sym = 0);
size_t gram_partials_cap(int c, int sm_count);
// Z (n x c2, ldz) = X (n x c1, ldx) * W (c1 x c2, ldw)
int gemm_nn(const double* X, int64_t ldx, const double* W, int64_t ldw, double* Z, int64_t ldz,
            int64_t n, int c1, int c2, cudaStream_t s, int upper = 0);
// Orthogonalization X (n x c) = Q (n x c', ld c') R (c' x c, row-major); see dense.cu.
// deflate = 0 tries CholeskyQR2 first and falls back to the deflated form when
// X is too ill-conditioned for it. ints: 8 device ints of scratch (8-byte aligned).
// The orthonormal factor is returned implicitly: on exit Q holds Q' (n x c') and, when
// Rcorr is not null, Rcorr holds the upper-triangular c' x c' matrix C with Q = Q' C.
// With Rcorr null only R is wanted (Q is then scratch of n x c doubles). r_from_gram (only
// with Rcorr null and deflate 0): when the plain Cholesky of X^T X succeeds, return its
// factor as R; the caller has checked that the Gram's rounding error is small enough.
size_t orth_scratch(int c, int64_t n, int sm_count);
int orth_qr(const double* X, int64_t ldx, int64_t n, int c, double* Q, double* R, int* c_out, double* scratch, int* ints,
            int deflate, cmsvd_context* ctx, double* Rcorr, bool r_from_gram = false);
// One-sided Jacobi SVD of Bm (brows x bcols, row-major). trans = 0 rotates the columns of
// Bm: Bm V = Xc (column-major brows x bcols), V bcols x bcols. trans = 1 rotates the
// columns of Bm^T: Bm^T V = Xc (column-major bcols x brows), V brows x brows holds the
// left singular vectors of Bm. sv_j = ||Xc_j||, perm sorts sv descending.
// flag2: 16 bytes of device scratch (8-byte aligned + 8).
// tol > 0 overrides the rotation threshold max(1e-15, rows u) (loose sweeps for the deflation).
// jac_ctl: jacobi_scratch_words(d) device words, d >= both dimensions (256-byte aligned):
// control words and the mailbox of the cooperative sweeps.
size_t jacobi_scratch_words(int d);
int jacobi_svd(const double* Bm, int brows, int bcols, int trans, double* Xc, double* V, double* sv, int* perm,
               int* flag2, cmsvd_context* ctx, double tol, unsigned* jac_ctl);

}  // namespace cmsvd
