/*
 * cmsvd -- complex moment-based interior SVD on one GPU (C ABI).
 *
 * Computes the singular triplets (sigma_i, u_i, v_i) of a real sparse m x n
 * matrix A whose singular values lie in [a, b] (problem statement, Sec. 1,
 * Eq. psvd), with the block SS-SVD method (Alg. 1) or its variant with the
 * nonlinear transformation z = exp(t) (Alg. 2).
 *
 * Conventions for every call:
 *   - Every call returns an int status (cmsvd_status); 0 is success. No C++
 *     exception crosses this boundary. cmsvd_last_error() gives a message.
 *   - "device" pointers are CUDA device addresses on the context's device;
 *     "host" pointers are ordinary host memory. Calls marked "any" accept
 *     either (the copy direction is inferred by CUDA unified addressing).
 *   - Dense blocks are row-major with the leading dimension equal to the
 *     number of columns unless stated otherwise. Triplet outputs are
 *     column-major (one contiguous vector per triplet).
 *   - All work of one context is ordered on that context's stream. Calls that
 *     return host-visible values synchronize that stream before returning.
 *   - A call on a context makes the context's device current while it runs and
 *     makes the caller's current device current again before it returns.
 *   - The library owns the objects it creates (context, matrix, result) until
 *     the matching destroy call. It never frees caller memory.
 */
#ifndef CMSVD_H
#define CMSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cmsvd_status {
    CMSVD_OK = 0,
    CMSVD_INVALID_ARG = 1,          /* a parameter is out of range (message says which) */
    CMSVD_INVALID_MATRIX = 2,       /* CSR structure or values rejected by validation */
    CMSVD_OUT_OF_MEMORY = 3,        /* a library allocation failed */
    CMSVD_WORKSPACE_TOO_SMALL = 4,  /* ws_bytes below cmsvd_workspace_size() */
    CMSVD_NOT_CONVERGED = 5,        /* a shifted solve hit max_iter; the result is still returned */
    CMSVD_BREAKDOWN = 6,            /* NaN/Inf in a recurrence or a non-positive Cholesky pivot */
    CMSVD_SUBSPACE_SATURATED = 7,   /* warning: numerical rank of S^ equals L*M (Thm. 1: t may exceed L*M) */
    CMSVD_CUDA_ERROR = 8,           /* a CUDA runtime call failed */
    CMSVD_NOT_SUPPORTED = 9,        /* valid request outside what this library implements */
    CMSVD_PENDING = 10              /* serving: the request has not finished yet */
} cmsvd_status;

typedef enum cmsvd_variant {
    CMSVD_LINEAR = 0,   /* Alg. 1: shifts z_j on the ellipse around [a^2, b^2] */
    CMSVD_NT = 1        /* Alg. 2: shifts exp(t_j), t_j on the ellipse around [2 ln a, 2 ln b]; needs a > 0 */
} cmsvd_variant;

typedef enum cmsvd_solver {
    CMSVD_SOLVER_AUTO = 0,    /* DIRECT when every connected component of A^T A is small, else DENSE when
                                 n <= 1024, else KRYLOV */
    CMSVD_SOLVER_KRYLOV = 1,  /* shifted COCG in two-pass Lanczos form, all shifts share one Krylov space */
    CMSVD_SOLVER_DIRECT = 2,  /* exact solves on each connected component of A^T A through its
                                 eigendecomposition (the paper solves directly, Sec. 4) */
    CMSVD_SOLVER_DENSE = 3    /* n <= 1024: A^T A formed densely and eigendecomposed once (one-sided Jacobi);
                                 every shifted solve and moment follows exactly from it */
} cmsvd_solver;

typedef enum cmsvd_precision {
    CMSVD_FP64 = 0,       /* every step in FP64 */
    CMSVD_MIXED = 1       /* Krylov solver on the FP32 pipe: A's values as stored (bf16, FP32, or FP64 split into
                             two FP32 parts), every Lanczos vector as a double-float pair hi + lo of FP32
                             numbers, SpMM, vector updates, dot products and the moment accumulation in
                             double-float arithmetic (error-free FP32 products and sums, unit roundoff ~2^-48).
                             The recurrence scalars (alpha, beta, LDL^T pivots, tridiagonal solves) and the
                             moments stay FP64, as do rank truncation and Rayleigh-Ritz. With refine > 0 every
                             shifted solve is then checked in FP64, R_j = X - (s_j I - A^T A) Y_j with FP64 A,
                             and refined by correction solves while ||R_j|| / ||X|| > tol_solve. The direct and
                             dense solvers ignore it. */
} cmsvd_precision;

/* Precision in which the library keeps A's values (cmsvd_csr_create). The values are rounded
   to it (round to nearest) when the matrix is created, so the stored matrix is the problem
   that every solve on it computes. FP64 steps read the stored values widened to FP64; the
   mixed-precision Krylov path streams them in their stored width (8, 4 or 2 bytes). */
typedef enum cmsvd_storage {
    CMSVD_STORE_FP64 = 0,
    CMSVD_STORE_FP32 = 1,
    CMSVD_STORE_BF16 = 2
} cmsvd_storage;

/* Method parameters. Names follow Alg. 1 / Alg. 2 and Sec. 4. */
typedef struct cmsvd_params {
    int32_t N;            /* quadrature points, even, 2..128 (N/2 systems are solved, Sec. 3.1) */
    int32_t L;            /* columns of V_in, 1..128 */
    int32_t M;            /* moments, 1 <= M <= N-1 (Prop. 1); L*M <= 512 */
    int32_t ell;          /* iteration technique count (Eqs. iter1-iter2), >= 1 */
    double delta;         /* rank threshold, relative to the largest singular value of S^ (default 1e-12) */
    double eps_tau;       /* spurious threshold on tau_i / sigma_S,1 (Sec. 3.4.2; default 1e-8) */
    double alpha;         /* ellipse aspect ratio (Sec. 4; default 0.1) */
    int32_t variant;      /* cmsvd_variant */
    int32_t solver;       /* cmsvd_solver */
    int32_t precision;    /* cmsvd_precision */
    int32_t max_iter;     /* Krylov iteration limit per pass (default 20000) */
    double tol_solve;     /* relative residual of every shifted solve, Krylov solver (default 1e-12) */
    double tol_triplet;   /* keep a triplet when ||A^T u - sigma v|| / ||A||_2 <= tol_triplet (default 1e-10) */
    double norm_A;        /* ||A||_2 if known; <= 0 lets the library estimate it by Lanczos */
    int32_t check_every;  /* Krylov iterations between host convergence checks (default 48) */
    int32_t direct_max_block; /* AUTO picks DIRECT when the largest component has at most this many columns (default 32) */
    int32_t profile;      /* 1: time every kernel class with CUDA events and fill the prof_* statistics (default 0) */
    int32_t refine;       /* Krylov solver: FP64 check of every shifted solve, R_j = X - (s_j I - A^T A) Y_j with
                             FP64 A, and up to this many rounds of correction solves (s_j I - A^T A) E_j = R_j,
                             Y_j += E_j, until max ||R_j|| / ||X|| <= tol_solve (default 0: no check) */
    int32_t estimate;     /* 1: also compute the residual estimate of Sec. 3.4.1 through S_+ = [S_1, ..., S_M]
                             (Eq. residual; NT: Eq. res_nonlinear with mu from one exact residual), returned by
                             cmsvd_result_copy_estimate. The exact residuals are always computed (default 0) */
    int32_t fault_breakdown_at; /* test hook, 0 = off: > 0 makes the Krylov solver treat column 0 as broken down
                             at that Lanczos step, as a non-finite coefficient would, so that the solve returns
                             CMSVD_BREAKDOWN (failure handling is tested without a real fault) */
} cmsvd_params;

/* Kernel classes of the prof_* statistics (index into the arrays). */
enum {
    CMSVD_PROF_SPMM = 0,        /* CSR SpMM with A or A^T outside the Krylov loop */
    CMSVD_PROF_KRYLOV = 1,      /* Lanczos passes (graph launches: SpMMs + vector kernels) */
    CMSVD_PROF_DIRECT = 2,      /* per-component direct solve + moments */
    CMSVD_PROF_GRAM = 3,        /* X^T Y of tall-skinny blocks */
    CMSVD_PROF_GEMM = 4,        /* tall-skinny X W */
    CMSVD_PROF_SMALL = 5,       /* Cholesky, triangular inverse, selection (one CTA) */
    CMSVD_PROF_OTHER = 6,       /* quadrature, norm estimate, norms, output copies */
    CMSVD_PROF_JACOBI = 7,      /* one-sided Jacobi SVDs of the small blocks */
    CMSVD_PROF_CLASSES = 8
};

/* Per-solve statistics. */
typedef struct cmsvd_stats {
    int64_t found;            /* t^, number of returned triplets */
    int64_t in_interval;      /* Ritz values phi_i in [a, b] before the tau and residual tests */
    int64_t rank;             /* columns kept by the delta truncation (Alg. 1 step 3) */
    int64_t krylov_iters;     /* Lanczos steps of the last filter application (0 for DIRECT) */
    int64_t max_component;    /* largest connected component of A^T A (DIRECT only) */
    int32_t solver_used;      /* cmsvd_solver actually run */
    int32_t converged;        /* 1 when every shifted solve met tol_solve */
    double norm_A;            /* ||A||_2 used for the residual normalisation */
    double sigma_S1;          /* largest singular value of S^ */
    double max_res_u;         /* max over returned triplets of ||A^T u - sigma v|| / ||A||_2 */
    double max_res_v;         /* max over returned triplets of ||A v - sigma u|| / ||A||_2 */
    double ms_solve;          /* Alg. 1 steps 1-2 (shifted solves + moments), GPU time */
    double ms_truncate;       /* step 3 */
    double ms_qr;             /* step 4 */
    double ms_ritz;           /* step 5, selection and residuals */
    int64_t kernel_launches;  /* kernels launched by this solve (graph nodes included) */
    int32_t refine_rounds;    /* refinement rounds run (last filter application) */
    int32_t pad_;
    double refine_residual;   /* max ||R_j|| / ||X|| after refinement (0 without refinement) */
    /* With params.profile = 1, per kernel class: event-timed GPU ms, launches, and the
       algorithmic bytes (compulsory DRAM traffic) and FP64 flops of those launches. */
    double prof_ms[CMSVD_PROF_CLASSES];
    int64_t prof_launches[CMSVD_PROF_CLASSES];
    double prof_bytes[CMSVD_PROF_CLASSES];
    double prof_flops[CMSVD_PROF_CLASSES];
    double ms_components;     /* host ms spent by this solve building the connected components of A^T A
                                 (solver AUTO, first solve on a matrix only; 0 otherwise). This symbolic
                                 set-up copies the CSR to the host and runs a union-find */
} cmsvd_stats;

typedef struct cmsvd_context cmsvd_context;
typedef struct cmsvd_matrix cmsvd_matrix;
typedef struct cmsvd_result cmsvd_result;

/* Static text for a status code. */
const char* cmsvd_status_string(int status);
/* Message of the last failing call on this thread (static storage, overwritten by the next failure). */
const char* cmsvd_last_error(void);
/* Fill *p with the defaults listed in cmsvd_params. Returns CMSVD_INVALID_ARG for NULL. */
int cmsvd_params_default(cmsvd_params* p);

/*
 * Context: binds the current CUDA device and a caller stream (cudaStream_t
 * passed as void*; NULL means the legacy default stream). The stream is
 * borrowed, not owned. The library also creates one internal stream of its
 * own for graph capture; work on it is ordered after and before the caller's
 * stream by events, so callers only ever synchronize their own stream. This
 * holds on error returns too: the caller's stream waits for whatever the failed
 * call had already queued.
 */
int cmsvd_context_create(void* stream, cmsvd_context** out);
int cmsvd_context_destroy(cmsvd_context* ctx);   /* NULL is accepted */

/*
 * Arithmetic of the tall dense products of the rank truncation and of qr(A V~) (Alg. 1 steps
 * 3-4: Grams X^T Y and products X W with n >= 16384 rows and 32..1024 columns) on this context.
 * mode 0 (default): FP64-accurate emulation on the BF16 tensor cores. Every FP64 operand is cut
 * into 8 slices of 7 bits (integers below 128, exact in bf16) under a power-of-two scale per
 * row or column; the slice products are BF16 GEMMs with FP32 accumulation, exact because every
 * sum of at most 1024 such products stays below 2^24, and they are added in FP64 per level of
 * equal scale. Each result is within a few 2^-53 of the products of the largest entries that
 * share its scales. mode 1: the FP64 pipe only. The paper computes these steps in FP64
 * (MATLAB svd and qr); this is a property of the implementation. CMSVD_INVALID_ARG otherwise.
 */
int cmsvd_context_set_dense_arith(cmsvd_context* ctx, int32_t mode);

/*
 * Sparse matrix A (m x n, m >= 1, n >= 1) in CSR form (the problem's A, Sec. 1, Eq. psvd).
 * rowptr: int64[m+1], colidx: int32[nnz], vals: float64[nnz]; where = 0 for host arrays, 1 for
 * device arrays. The library copies them into its own device memory (the caller keeps
 * ownership of its arrays), validates them on the device (rowptr monotone from 0 to nnz,
 * columns strictly increasing within a row and in [0, n), values finite: otherwise
 * CMSVD_INVALID_MATRIX and *out is NULL), rounds the values to `storage` (cmsvd_storage;
 * CMSVD_INVALID_MATRIX if one overflows it) and builds the CSR of A^T. The paper assumes
 * m >= n (Sec. 1); m < n is accepted and simply means A^T A is rank deficient.
 */
int cmsvd_csr_create(cmsvd_context* ctx, int64_t m, int64_t n, int64_t nnz,
                     const int64_t* rowptr, const int32_t* colidx, const double* vals,
                     int where, int32_t storage, cmsvd_matrix** out);
int cmsvd_csr_destroy(cmsvd_matrix* A);          /* NULL is accepted */
/* Dimensions of A. */
int cmsvd_csr_shape(const cmsvd_matrix* A, int64_t* m, int64_t* n, int64_t* nnz);

/*
 * Y = A X (transpose = 0, X n x L, Y m x L) or Y = A^T X (transpose = 1,
 * X m x L, Y n x L); device pointers, row-major with leading dimensions
 * ldx >= L and ldy >= L. This is the H X = A^T (A X) building block of every
 * shifted solve (Alg. 1 steps 1-2) and of A V~ (step 4).
 */
int cmsvd_spmm(cmsvd_matrix* A, int transpose, int64_t L, const double* X, int64_t ldx,
               double* Y, int64_t ldy);

/*
 * The same product in FP32, the SpMM of the mixed-precision Krylov path: FP32 values of A
 * (a copy made on the device at the first call and kept with the matrix), FP32 X and Y,
 * FP32 accumulation in each row's storage order. Layouts and errors as cmsvd_spmm.
 */
int cmsvd_spmm_f32(cmsvd_matrix* A, int transpose, int64_t L, const float* X, int64_t ldx,
                   float* Y, int64_t ldy);

/*
 * The same product in double-float arithmetic, the SpMM of the mixed-precision Krylov path
 * (Alg. 1 steps 1-2). X and Y are device blocks of FP32 pairs: row i holds the L high parts
 * x_hi[i, 0..L-1] followed by the L low parts x_lo[i, 0..L-1], the value being x_hi + x_lo;
 * ldx, ldy >= 2L are in floats. Products a * x_hi are formed exactly and the sums are
 * compensated, all on the FP32 pipe, so Y = A X to a few units of 2^-48 of sum |a||x| (FP32
 * or bf16 values are exact; FP64 values that are not FP32-exact are used as hi + lo FP32
 * pairs). Y is normalized (|y_lo| <= ulp(y_hi) / 2). Errors as cmsvd_spmm.
 */
int cmsvd_spmm_df(cmsvd_matrix* A, int transpose, int64_t L, const float* X, int64_t ldx,
                  float* Y, int64_t ldy);

/*
 * The SpMM autotuner's pick for A (transpose = 0) or A^T (transpose = 1), operand kind 0
 * (FP64, cmsvd_spmm), 1 (FP32, cmsvd_spmm_f32) or 2 (double-float, cmsvd_spmm_df) and width L.
 * The first product of a kind and width on a matrix through those entry points, and the first
 * Lanczos product of a Krylov solve (before its graph capture), times every kernel variant on
 * its own operands and keeps the fastest; all variants give bitwise equal results. Products
 * inside a solve's other steps use a kept pick or the default configuration and never tune.
 * cfg[4] (host) receives lanes per row, gathers in flight per lane, column slices per product,
 * and 1 when rows run in storage order (0: rows sorted by first column); *ms (may be NULL) the
 * time of one product in the tuning run. CMSVD_NOT_SUPPORTED when no pick exists yet. This is
 * a property of the implementation; the paper has none.
 */
int cmsvd_spmm_tuning(const cmsvd_matrix* A, int transpose, int32_t kind, int64_t L, int32_t* cfg, float* ms);

/*
 * Quadrature of Sec. 4 for j = 1..N/2 (the points with Im > 0, Sec. 3.1),
 * computed on the device. Outputs are host arrays of N/2 complex values,
 * interleaved (re, im): shift[j] = z_j (linear) or exp(t_j) (NT);
 * weight[j] = omega_j (linear) or psi_j (NT); scaled[j] = (z_j - gamma)/rho
 * (or (t_j - gamma)/rho), the node used for the moment weights. Any output
 * may be NULL.
 */
int cmsvd_quadrature(cmsvd_context* ctx, double a, double b, int32_t N, int32_t variant,
                     double alpha, double* shift, double* weight, double* scaled);

/*
 * G = X^T Y for tall-skinny device blocks: the Gram product of the CholeskyQR
 * orthogonalizations in the rank truncation (Alg. 1 step 3) and in qr(A V~)
 * (step 4). X: n x c1 (leading dimension ldx >= c1), Y: n x c2 (ldy >= c2),
 * G: c1 x c2 row-major; all device, all FP64. Deterministic: the rows are split
 * into fixed chunks whose partial products are added in chunk order. For n >= 16384 and
 * 32 <= c1 <= 1024, c2 >= 32 it follows the context's dense arithmetic
 * (cmsvd_context_set_dense_arith).
 * workspace: device scratch of at least cmsvd_gram_workspace_size bytes, owned by
 * the caller. 1 <= c1, c2 <= 4096, n >= 1.
 */
int cmsvd_gram_workspace_size(cmsvd_context* ctx, int64_t n, int32_t c1, int32_t c2, size_t* bytes);
int cmsvd_gram(cmsvd_context* ctx, int64_t n, int32_t c1, int32_t c2, const double* X, int64_t ldx,
               const double* Y, int64_t ldy, double* G, void* workspace, size_t ws_bytes);

/*
 * cmsvd_gram without a workspace argument, for callers that cannot allocate
 * device memory when they call: code whose device memory is all owned by
 * another allocator, real-time loops where a cudaMalloc would synchronize the
 * device, and host programs that hand a library only the buffers of the call.
 * The paper has no counterpart; this is a property of the library interface.
 *
 * Same arguments, limits (1 <= c1, c2 <= 4096) and result as cmsvd_gram (within rounding:
 * the chunking may differ), plus c1 * c2 <= 1,048,576: the chunk partials live in one fixed
 * 8 MiB array of device memory inside the library (1,048,576 doubles), held by every GPU that
 * loads the library until the process exits. Larger requests return CMSVD_INVALID_ARG. The
 * call allocates nothing. The first call on a device looks up the array's device address
 * (one-time set-up) and keeps it for the life of the process; make that first call before
 * any stream capture on that device, and do not call it after cudaDeviceReset or a release of
 * the device's primary context (the array then moves and the kept address is stale).
 * Every call shares the array: calls that overlap on the GPU (other streams, other contexts,
 * other threads) race and must be serialized by the caller. Like every entry point, it makes
 * the context's device current while it runs and restores the caller's current device.
 */
int cmsvd_gram_noalloc(cmsvd_context* ctx, int64_t n, int32_t c1, int32_t c2, const double* X, int64_t ldx,
                       const double* Y, int64_t ldy, double* G);

/*
 * Z = X W for a tall device block X (n x c1, ldx >= c1) and a small one W (c1 x c2, ldw >= c2),
 * Z n x c2 (ldz >= c2), all row-major FP64: the product that forms the orthonormal bases of the
 * rank truncation (Alg. 1 step 3) and the Ritz vectors (step 5). For n >= 16384 and
 * 32 <= c1 <= 1024, c2 >= 32 it follows the context's dense arithmetic
 * (cmsvd_context_set_dense_arith); with dense arithmetic 0, a product with c1 >= 128 and fewer
 * 64 x 64 output tiles than the GPU has SMs runs on cuBLAS's FP64 GEMM, which splits the
 * contraction over the GPU. Deterministic in every case. 1 <= c1, c2 <= 4096.
 */
int cmsvd_gemm(cmsvd_context* ctx, int64_t n, int32_t c1, int32_t c2, const double* X, int64_t ldx,
               const double* W, int64_t ldw, double* Z, int64_t ldz);

/* Device workspace (bytes) that cmsvd_moments / cmsvd_solve_interval need for A and *p. */
int cmsvd_workspace_size(const cmsvd_matrix* A, const cmsvd_params* p, size_t* bytes);

/*
 * Moment block of Alg. 1/2 steps 1-2 (with the halving of Sec. 3.1):
 *   S_k = 2 Re sum_{j<=N/2} w_j ((node_j - gamma)/rho)^k (s_j I - A^T A)^{-1} S_0^(ell-1),
 * k = 0..M (M+1 blocks: the last one is the S_M block of S_+, Sec. 3.4.1).
 * V_in: device, n x L. S_out: device, n x L(M+1) row-major, column m*L + l.
 * The moment weights use the scaled node (node_j - gamma)/rho in place of the
 * literal node^k of Sec. 3.1: the two moment blocks differ by a block-triangular
 * change of basis, so they span the same column space, and the scaled form keeps
 * the blocks well conditioned when rho << gamma. Returns CMSVD_NOT_CONVERGED
 * (with S_out filled) when a Krylov solve hit max_iter.
 */
int cmsvd_moments(cmsvd_matrix* A, double a, double b, const cmsvd_params* p,
                  const double* V_in, double* S_out, void* workspace, size_t ws_bytes,
                  cmsvd_stats* stats);

/*
 * Whole method, Alg. 1 (variant LINEAR) or Alg. 2 (variant NT): moments, rank
 * truncation with delta (step 3), QR of A V~ (step 4), SVD of B and Ritz
 * triplets (step 5), the tau test (Sec. 3.4.2) and exact residuals.
 * V_in: device n x L (caller-drawn, e.g. Gaussian). workspace: device,
 * >= cmsvd_workspace_size bytes, caller-owned; the result's arrays live in it,
 * so it must outlive the result. *out receives a library-owned result (also
 * on CMSVD_NOT_CONVERGED and CMSVD_SUBSPACE_SATURATED).
 */
int cmsvd_solve_interval(cmsvd_matrix* A, double a, double b, const cmsvd_params* p,
                         const double* V_in, void* workspace, size_t ws_bytes,
                         cmsvd_result** out);

/*
 * Residual estimate of Sec. 3.4.1 for every returned triplet (host or device memory, t
 * doubles), relative to ||A||_2 like res_u. With scaled moment nodes m_j = (zeta_j - gamma)/rho,
 * f(A^T A) S_k = rho S_{k+1} + gamma S_k (f(x) = x: Prop. 1, exact up to the solves; NT:
 * f(x) = ln x, Eq. sk=aks_nonlinear, approximate), so with v = U_S1 q = S W_S1 Sigma_S1^{-1} q
 *   r~_i = || rho S_+ W_S1 Sigma_S1^{-1} q_i + (gamma - f(sigma_i^2)) v_i || / sigma_i.
 * Linear variant: the estimate is r~_i / ||A||_2 (equal to res_u up to rounding and solve error).
 * NT: mu r~_i / ||A||_2 with mu = ||r_i'|| / ||r~_i'|| (Eq. res_nonlinear); i' is the candidate
 * (sigma in [a, b], not spurious) with the largest r~ (the paper leaves i' open).
 * CMSVD_NOT_SUPPORTED when the solve ran with estimate = 0.
 */
int cmsvd_result_copy_estimate(const cmsvd_result* r, double* res_est);

/*
 * Batched solves (no counterpart in the paper, which solves one problem at a time):
 * count independent problems, problem i being cmsvd_solve_interval(A[i], a[i], b[i], &p[i],
 * V_in[i], workspace[i], ws_bytes[i], &out[i]). Problems whose matrices share a context run
 * one after another, in index order, on that context's stream. Problems on different
 * contexts run concurrently, one host thread per context. To overlap many small problems,
 * create several contexts and spread the matrices over them. Each problem needs its own
 * workspace, because its result lives there until cmsvd_result_destroy. Results are
 * identical to solving each problem alone.
 * status[i] receives each problem's status and out[i] its result (NULL when it failed).
 * Returns CMSVD_OK when every status is OK, NOT_CONVERGED or SUBSPACE_SATURATED. Otherwise
 * it returns the first failing status, and cmsvd_last_error names the problem.
 */
int cmsvd_solve_batch(int count, cmsvd_matrix* const* A, const double* a, const double* b,
                      const cmsvd_params* p, const double* const* V_in, void* const* workspace,
                      const size_t* ws_bytes, cmsvd_result** out, int* status);

/*
 * Serving loop with continuous batching. The paper has no counterpart; it solves one
 * problem at a time. A server owns `slots` contexts, each with its own stream and host
 * worker thread, and a set of resident matrices.
 * - Requests are interval-SVD solves on a resident matrix with host V_in. They queue in
 *   arrival order.
 * - The head request is admitted as soon as a slot is free and its workspace fits in the
 *   HBM budget left after the resident matrices and the running requests. Admitted
 *   requests run concurrently.
 * - Each result is copied to host memory when its solve completes. It is identical to
 *   solving the request alone with cmsvd_solve_interval.
 * hbm_budget = 0 takes 80% of the free device memory at creation.
 * Latency is measured from submit to result ready, and queueing from submit to admission.
 */
typedef struct cmsvd_server cmsvd_server;
int cmsvd_server_create(int slots, size_t hbm_budget, cmsvd_server** out);
/* Stops the workers (a running solve finishes first); requests not started are dropped.
 * Call it only after every cmsvd_server_wait on this server has returned. */
int cmsvd_server_destroy(cmsvd_server* s);
/* Uploads, validates and registers a matrix (as cmsvd_csr_create, with the same storage
 * argument); *id names it in requests.
 * Safe to call while requests run. CMSVD_OUT_OF_MEMORY (nothing registered) when the matrix
 * does not fit in the budget beside the resident matrices and the largest queued request. */
int cmsvd_server_add_matrix(cmsvd_server* s, int64_t m, int64_t n, int64_t nnz, const int64_t* rowptr,
                            const int32_t* colidx, const double* vals, int vals_on_device, int32_t storage,
                            int* id);
/* Queues a request; V_in (n x L, row-major, host memory) is copied. Returns at once with a
 * ticket. CMSVD_OUT_OF_MEMORY when its workspace can never fit in the budget. */
int cmsvd_server_submit(cmsvd_server* s, int id, double a, double b, const cmsvd_params* p,
                        const double* V_in_host, int64_t* ticket);
/* Waits up to timeout_ms (< 0: forever) for a request. CMSVD_PENDING if it has not finished;
 * otherwise CMSVD_OK, with t = triplets found, solve_status = the solve's own status, and the
 * latency and queueing times in ms (any output pointer may be NULL). */
int cmsvd_server_wait(cmsvd_server* s, int64_t ticket, int timeout_ms, int64_t* t, int* solve_status,
                      double* latency_ms, double* queue_ms);
/* Copies a finished request's triplets to host buffers that hold `capacity` triplets
 * (layouts of cmsvd_result_copy; any pointer may be NULL) and forgets the request.
 * CMSVD_INVALID_ARG (nothing copied, request kept) when capacity < t. */
int cmsvd_server_take(cmsvd_server* s, int64_t ticket, int64_t capacity, double* sigma, double* U, double* V,
                      double* res_u, double* res_v, double* tau, cmsvd_stats* stats);

/* Number of triplets found (t^). */
int cmsvd_result_count(const cmsvd_result* r, int64_t* t);
/*
 * Copy the triplets (any memory; each pointer may be NULL): sigma[t] ascending;
 * U m x t and V n x t column-major; res_u[t] = ||A^T u - sigma v|| / ||A||_2;
 * res_v[t] = ||A v - sigma u|| / ||A||_2; tau[t] = tau_i / sigma_S,1.
 * Signs: the largest-magnitude entry of each v (first on ties) is positive.
 */
int cmsvd_result_copy(const cmsvd_result* r, double* sigma, double* U, double* V,
                      double* res_u, double* res_v, double* tau);
int cmsvd_result_stats(const cmsvd_result* r, cmsvd_stats* stats);
int cmsvd_result_destroy(cmsvd_result* r);       /* NULL is accepted */

#ifdef __cplusplus
}
#endif
#endif /* CMSVD_H */
