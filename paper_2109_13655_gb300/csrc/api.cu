// C-ABI entry points (include/cmsvd.h) and the orchestration of one solve.
#include "internal.cuh"
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <new>

namespace cmsvd {
const char* last_error();
size_t ritz_workspace(int64_t m, int64_t n, int c, int sm_count);
int rayleigh_ritz(cmsvd_matrix* M, const double* S, int64_t lds, int c, double a, double b, const cmsvd_params* p,
                  double normA, Arena& ws, const RitzOut& out, cmsvd_stats* st, cudaEvent_t* ev);
}  // namespace cmsvd

using namespace cmsvd;

namespace {

struct Events {
    cudaEvent_t e[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    ~Events() {
        for (auto& x : e)
            if (x) cudaEventDestroy(x);
    }
    int make() {
        for (auto& x : e) CM_CUDA(cudaEventCreate(&x));
        return CMSVD_OK;
    }
};

int check_params(const cmsvd_matrix* A, double a, double b, const cmsvd_params* p) {
    if (!A || !p) { set_error("NULL matrix or params"); return CMSVD_INVALID_ARG; }
    if (!(a >= 0.0) || !(b > a) || !std::isfinite(b)) { set_error("need 0 <= a < b (got a=%g b=%g)", a, b); return CMSVD_INVALID_ARG; }
    if (p->N < 2 || p->N > 128 || (p->N & 1)) { set_error("N must be even in [2, 128] (got %d)", p->N); return CMSVD_INVALID_ARG; }
    if (p->L < 1 || p->L > 128) { set_error("L must be in [1, 128] (got %d)", p->L); return CMSVD_INVALID_ARG; }
    if (p->M < 1 || p->M > p->N - 1) { set_error("M must be in [1, N-1] (got %d)", p->M); return CMSVD_INVALID_ARG; }
    if ((int64_t)p->L * p->M > 512) { set_error("L*M must be <= 512 (got %d)", p->L * p->M); return CMSVD_INVALID_ARG; }
    if (p->ell < 1) { set_error("ell must be >= 1"); return CMSVD_INVALID_ARG; }
    if (p->variant != CMSVD_LINEAR && p->variant != CMSVD_NT) { set_error("unknown variant %d", p->variant); return CMSVD_INVALID_ARG; }
    if (p->variant == CMSVD_NT && !(a > 0.0)) { set_error("the exp transform (NT variant) needs a > 0"); return CMSVD_INVALID_ARG; }
    if (!(p->alpha > 0.0)) { set_error("alpha must be > 0"); return CMSVD_INVALID_ARG; }
    if (p->max_iter < 1) { set_error("max_iter must be >= 1"); return CMSVD_INVALID_ARG; }
    if (p->refine < 0 || p->refine > 100) { set_error("refine must be in [0, 100]"); return CMSVD_INVALID_ARG; }
    if (p->estimate != 0 && p->estimate != 1) { set_error("estimate must be 0 or 1"); return CMSVD_INVALID_ARG; }
    if (p->fault_breakdown_at < 0) { set_error("fault_breakdown_at must be >= 0"); return CMSVD_INVALID_ARG; }
    if (!(p->delta >= 0.0) || !(p->eps_tau >= 0.0) || !(p->tol_triplet > 0.0) || !(p->tol_solve > 0.0)) {
        set_error("delta, eps_tau >= 0 and tol_solve, tol_triplet > 0 required");
        return CMSVD_INVALID_ARG;
    }
    if (p->solver < CMSVD_SOLVER_AUTO || p->solver > CMSVD_SOLVER_DENSE) { set_error("unknown solver %d", p->solver); return CMSVD_INVALID_ARG; }
    if (p->solver == CMSVD_SOLVER_DENSE && A->A.n > 1024) { set_error("the DENSE solver needs n <= 1024"); return CMSVD_INVALID_ARG; }
    if (p->precision != CMSVD_FP64 && p->precision != CMSVD_MIXED) { set_error("unknown precision %d", p->precision); return CMSVD_INVALID_ARG; }
    if ((int64_t)p->L * p->M > A->A.n) {
        set_error("L*M (%d) exceeds n (%lld)", p->L * p->M, (long long)A->A.n);
        return CMSVD_INVALID_ARG;
    }
    return CMSVD_OK;
}

// AUTO: the connected components of A^T A decide (built once per matrix, on the host: the
// symbolic phase of the direct solve, timed into stats->ms_components). Errors propagate.
int pick_solver(cmsvd_matrix* A, const cmsvd_params* p, int* solver, cmsvd_stats* st) {
    if (p->solver != CMSVD_SOLVER_AUTO) { *solver = p->solver; return CMSVD_OK; }
    if (!A->comp.ready) {
        const auto t0 = std::chrono::steady_clock::now();
        CM_TRY(components_build(A));
        A->ms_components = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        st->ms_components = A->ms_components;
    }
    if (A->comp.max_size <= p->direct_max_block) *solver = CMSVD_SOLVER_DIRECT;
    else *solver = A->A.n <= 1024 ? CMSVD_SOLVER_DENSE : CMSVD_SOLVER_KRYLOV;
    return CMSVD_OK;
}

// Workspace plan shared by the size query and the solve.
struct Plan {
    double2* quad;
    double* S;
    RitzOut out;
    size_t persistent;
};

void plan_persistent(Arena& ws, const cmsvd_matrix* A, const cmsvd_params* p, Plan& pl, bool with_outputs) {
    const int J = p->N / 2, c = p->L * p->M;
    pl.quad = ws.take<double2>(3 * (size_t)J);
    pl.S = ws.take<double>((size_t)A->A.n * p->L * (p->M + 1));
    if (with_outputs) {
        pl.out.sigma = ws.take<double>(c);
        pl.out.U = ws.take<double>((size_t)A->A.m * c);
        pl.out.V = ws.take<double>((size_t)A->A.n * c);
        pl.out.res_u = ws.take<double>(c);
        pl.out.res_v = ws.take<double>(c);
        pl.out.tau = ws.take<double>(c);
        pl.out.res_est = ws.take<double>(c);
    }
    pl.persistent = ws.off;
}

size_t scratch_size(const cmsvd_matrix* A, const cmsvd_params* p, bool with_ritz) {
    size_t mx = krylov_workspace(A, p);
    size_t d = direct_workspace(A, p);
    if (d > mx) mx = d;
    d = dense_workspace(A, p);
    if (d > mx) mx = d;
    if (with_ritz) {
        size_t r = ritz_workspace(A->A.m, A->A.n, p->L * p->M, A->ctx->sm_count);
        if (r > mx) mx = r;
    }
    // norm estimate: Lanczos with one column and 128 steps
    cmsvd_params q = *p;
    q.L = 1; q.N = 2; q.M = 0; q.max_iter = 128;
    size_t ne = krylov_workspace(A, &q) + sizeof(double) * (A->A.n + 64);
    if (ne > mx) mx = ne;
    return mx;
}

int ensure_norm(cmsvd_matrix* A, const cmsvd_params* p, Arena& ws, double* normA) {
    if (p->norm_A > 0.0) { *normA = p->norm_A; return CMSVD_OK; }
    if (A->norm_est <= 0.0) {
        size_t mark = ws.off;
        CM_TRY(norm_estimate(A, ws, &A->norm_est));
        ws.off = mark;
    }
    *normA = A->norm_est;
    return CMSVD_OK;
}

// Steps 1-2 into pl.S. Returns the solve status (OK or NOT_CONVERGED) or an error.
int run_moments(cmsvd_matrix* A, double a, double b, const cmsvd_params* p, const double* V_in, Plan& pl, Arena& ws,
                cmsvd_stats* st) {
    cmsvd_context* ctx = A->ctx;
    QuadParams qp{a, b, p->alpha, p->N, p->variant};
    CM_TRY(quadrature_device(qp, pl.quad, ctx->s));
    int solver = CMSVD_SOLVER_AUTO;
    CM_TRY(pick_solver(A, p, &solver, st));
    st->solver_used = solver;
    const int64_t lds = (int64_t)p->L * (p->M + 1);
    size_t mark = ws.off;
    int status = CMSVD_OK;
    if (solver == CMSVD_SOLVER_DIRECT) {
        CM_TRY(direct_moments(A, p, pl.quad, p->M + 1, V_in, p->L, pl.S, lds, ws));
        st->converged = 1;
        st->krylov_iters = 0;
        st->max_component = A->comp.max_size;
    } else if (solver == CMSVD_SOLVER_DENSE) {
        CM_TRY(dense_moments(A, p, pl.quad, p->M + 1, V_in, p->L, pl.S, lds, ws));
        st->converged = 1;
        st->krylov_iters = 0;
        st->max_component = A->comp.ready ? A->comp.max_size : A->A.n;
    } else {
        SolveOut so;
        CM_TRY(krylov_moments(A, p, pl.quad, p->M + 1, V_in, p->L, pl.S, lds, ws, &so));
        st->krylov_iters = so.iters;
        st->converged = so.converged;
        st->refine_rounds = so.refine_rounds;
        st->refine_residual = so.refine_residual;
        if (!so.converged) status = CMSVD_NOT_CONVERGED;
    }
    ws.off = mark;
    return status;
}

}  // namespace

// ============================================================================= exported
extern "C" {

const char* cmsvd_status_string(int status) {
    switch (status) {
        case CMSVD_OK: return "ok";
        case CMSVD_INVALID_ARG: return "invalid argument";
        case CMSVD_INVALID_MATRIX: return "invalid matrix";
        case CMSVD_OUT_OF_MEMORY: return "out of memory";
        case CMSVD_WORKSPACE_TOO_SMALL: return "workspace too small";
        case CMSVD_NOT_CONVERGED: return "not converged";
        case CMSVD_BREAKDOWN: return "breakdown";
        case CMSVD_SUBSPACE_SATURATED: return "subspace saturated";
        case CMSVD_CUDA_ERROR: return "CUDA error";
        case CMSVD_NOT_SUPPORTED: return "not supported";
        case CMSVD_PENDING: return "pending";
        default: return "unknown status";
    }
}

const char* cmsvd_last_error(void) { return cmsvd::last_error(); }

int cmsvd_params_default(cmsvd_params* p) {
    if (!p) { set_error("NULL params"); return CMSVD_INVALID_ARG; }
    p->N = 32;
    p->L = 16;
    p->M = 4;
    p->ell = 1;
    p->delta = 1e-12;
    p->eps_tau = 1e-8;
    p->alpha = 0.1;
    p->variant = CMSVD_LINEAR;
    p->solver = CMSVD_SOLVER_AUTO;
    p->precision = CMSVD_FP64;
    p->max_iter = 20000;
    p->tol_solve = 1e-12;
    p->tol_triplet = 1e-10;
    p->norm_A = 0.0;
    p->check_every = 48;
    p->direct_max_block = 32;
    p->profile = 0;
    p->refine = 0;
    p->estimate = 0;
    p->fault_breakdown_at = 0;
    return CMSVD_OK;
}

int cmsvd_context_create(void* stream, cmsvd_context** out) {
    if (!out) { set_error("NULL out"); return CMSVD_INVALID_ARG; }
    *out = nullptr;
    cmsvd_context* c = new (std::nothrow) cmsvd_context();
    if (!c) { set_error("host allocation failed"); return CMSVD_OUT_OF_MEMORY; }
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&c->pinned, 256);
    if (e != cudaSuccess) {
        int st = cuda_fail(e, "context create", __FILE__, __LINE__);
        cmsvd_context_destroy(c);
        return st;
    }
    c->user = (cudaStream_t)stream;
    *out = c;
    return CMSVD_OK;
}

int cmsvd_context_destroy(cmsvd_context* c) {
    if (!c) return CMSVD_OK;
    if (c->s) cudaStreamSynchronize(c->s);
    ozaki_release(c);
    if (c->s) cudaStreamDestroy(c->s);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->pinned) cudaFreeHost(c->pinned);
    delete c;
    return CMSVD_OK;
}

int cmsvd_context_set_dense_arith(cmsvd_context* ctx, int32_t mode) {
    if (!ctx) { set_error("NULL context"); return CMSVD_INVALID_ARG; }
    if (mode != 0 && mode != 1) { set_error("mode must be 0 (tensor-core FP64 emulation) or 1 (FP64 pipe)"); return CMSVD_INVALID_ARG; }
    ctx->dense_arith = mode;
    return CMSVD_OK;
}

int cmsvd_csr_create(cmsvd_context* ctx, int64_t m, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                     const double* vals, int where, int32_t storage, cmsvd_matrix** out) {
    if (!out) { set_error("NULL out"); return CMSVD_INVALID_ARG; }
    *out = nullptr;
    if (!ctx) { set_error("NULL context"); return CMSVD_INVALID_ARG; }
    if (m < 1 || n < 1 || nnz < 0 || m >= (int64_t(1) << 31) || n >= (int64_t(1) << 31)) {
        set_error("need 1 <= m, n < 2^31 and nnz >= 0 (m=%lld n=%lld nnz=%lld)", (long long)m, (long long)n, (long long)nnz);
        return CMSVD_INVALID_ARG;
    }
    if (!rowptr || (nnz > 0 && (!colidx || !vals))) { set_error("NULL CSR array"); return CMSVD_INVALID_ARG; }
    if (storage != CMSVD_STORE_FP64 && storage != CMSVD_STORE_FP32 && storage != CMSVD_STORE_BF16) {
        set_error("unknown storage %d", storage);
        return CMSVD_INVALID_ARG;
    }
    Session se;
    CM_TRY(se.open(ctx));
    cmsvd_matrix* M = new (std::nothrow) cmsvd_matrix();
    if (!M) { set_error("host allocation failed"); return CMSVD_OUT_OF_MEMORY; }
    M->ctx = ctx;
    int st = csr_upload_validate(ctx, m, n, nnz, rowptr, colidx, vals, where, &M->A);
    if (st == CMSVD_OK) st = csr_round_storage(ctx, &M->A, storage);
    if (st == CMSVD_OK) st = csr_transpose(ctx, M->A, &M->At);
    if (st == CMSVD_OK) st = csr_round_storage(ctx, &M->At, storage);   // values already rounded: keeps the bf16 copy
    if (st != CMSVD_OK) {
        csr_free(&M->A);
        csr_free(&M->At);
        delete M;
        return st;
    }
    CM_TRY(se.close());
    *out = M;
    return CMSVD_OK;
}

int cmsvd_csr_destroy(cmsvd_matrix* A) {
    if (!A) return CMSVD_OK;
    cudaStreamSynchronize(A->ctx->s);
    csr_free(&A->A);
    csr_free(&A->At);
    components_free(&A->comp);
    delete A;
    return CMSVD_OK;
}

int cmsvd_csr_shape(const cmsvd_matrix* A, int64_t* m, int64_t* n, int64_t* nnz) {
    if (!A) { set_error("NULL matrix"); return CMSVD_INVALID_ARG; }
    if (m) *m = A->A.m;
    if (n) *n = A->A.n;
    if (nnz) *nnz = A->A.nnz;
    return CMSVD_OK;
}

int cmsvd_spmm(cmsvd_matrix* A, int transpose, int64_t L, const double* X, int64_t ldx, double* Y, int64_t ldy) {
    if (!A || !X || !Y) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    if (L < 1 || L > 4096 || ldx < L || ldy < L) { set_error("need 1 <= L <= 4096, ldx >= L, ldy >= L"); return CMSVD_INVALID_ARG; }
    Session se;
    CM_TRY(se.open(A->ctx));
    CM_TRY(spmm_tune(transpose ? A->At : A->A, SPMM_KIND_F64, (int)L, X, ldx, Y, ldy, A->ctx->s));
    return se.close();
}

int cmsvd_spmm_f32(cmsvd_matrix* A, int transpose, int64_t L, const float* X, int64_t ldx, float* Y, int64_t ldy) {
    if (!A || !X || !Y) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    if (L < 1 || L > 4096 || ldx < L || ldy < L) { set_error("need 1 <= L <= 4096, ldx >= L, ldy >= L"); return CMSVD_INVALID_ARG; }
    Session se;
    CM_TRY(se.open(A->ctx));
    CM_TRY(csr_make_fp32(A));
    CM_TRY(spmm_tune(transpose ? A->At : A->A, SPMM_KIND_F32, (int)L, X, ldx, Y, ldy, A->ctx->s));
    return se.close();
}

int cmsvd_spmm_df(cmsvd_matrix* A, int transpose, int64_t L, const float* X, int64_t ldx, float* Y, int64_t ldy) {
    if (!A || !X || !Y) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    if (L < 1 || L > 4096 || ldx < 2 * L || ldy < 2 * L) { set_error("need 1 <= L <= 4096, ldx >= 2L, ldy >= 2L"); return CMSVD_INVALID_ARG; }
    Session se;
    CM_TRY(se.open(A->ctx));
    CM_TRY(csr_make_fp32(A));
    CM_TRY(spmm_tune(transpose ? A->At : A->A, SPMM_KIND_DF, (int)L, X, ldx, Y, ldy, A->ctx->s));
    return se.close();
}

int cmsvd_spmm_tuning(const cmsvd_matrix* A, int transpose, int32_t kind, int64_t L, int32_t* cfg, float* ms) {
    if (!A || !cfg) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    if (kind < 0 || kind > 2) { set_error("kind must be 0 (FP64), 1 (FP32) or 2 (double-float)"); return CMSVD_INVALID_ARG; }
    SpmmCfg c;
    if (!spmm_tuned(transpose ? A->At : A->A, kind, (int)L, &c)) {
        set_error("no autotuned configuration for this matrix, kind and L yet");
        return CMSVD_NOT_SUPPORTED;
    }
    cfg[0] = c.lpr;
    cfg[1] = c.unroll;
    cfg[2] = c.slices;
    cfg[3] = c.natural;
    if (ms) *ms = c.ms;
    return CMSVD_OK;
}

int cmsvd_quadrature(cmsvd_context* ctx, double a, double b, int32_t N, int32_t variant, double alpha, double* shift,
                     double* weight, double* scaled) {
    if (!ctx) { set_error("NULL context"); return CMSVD_INVALID_ARG; }
    if (!(a >= 0.0) || !(b > a) || N < 2 || N > 128 || (N & 1) || !(alpha > 0.0) ||
        (variant != CMSVD_LINEAR && variant != CMSVD_NT) || (variant == CMSVD_NT && !(a > 0.0))) {
        set_error("invalid quadrature arguments");
        return CMSVD_INVALID_ARG;
    }
    Session se;
    CM_TRY(se.open(ctx));
    const int J = N / 2;
    double2* d = nullptr;
    CM_CUDA(cudaMalloc(&d, sizeof(double2) * 3 * J));
    QuadParams q{a, b, alpha, N, variant};
    int st = quadrature_device(q, d, ctx->s);
    double2* h = (double2*)malloc(sizeof(double2) * 3 * J);
    if (st == CMSVD_OK && h) {
        cudaError_t e = cudaMemcpyAsync(h, d, sizeof(double2) * 3 * J, cudaMemcpyDeviceToHost, ctx->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
        if (e != cudaSuccess) st = cuda_fail(e, "quadrature copy", __FILE__, __LINE__);
    }
    if (st == CMSVD_OK && h) {
        for (int j = 0; j < J; ++j) {
            if (shift) { shift[2 * j] = h[3 * j].x; shift[2 * j + 1] = h[3 * j].y; }
            if (weight) { weight[2 * j] = h[3 * j + 1].x; weight[2 * j + 1] = h[3 * j + 1].y; }
            if (scaled) { scaled[2 * j] = h[3 * j + 2].x; scaled[2 * j + 1] = h[3 * j + 2].y; }
        }
    }
    free(h);
    cudaFree(d);
    if (st != CMSVD_OK) return st;
    return se.close();
}

int cmsvd_gram_workspace_size(cmsvd_context* ctx, int64_t n, int32_t c1, int32_t c2, size_t* bytes) {
    if (!ctx || !bytes) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    if (n < 1 || c1 < 1 || c2 < 1 || c1 > 4096 || c2 > 4096) { set_error("need n >= 1 and 1 <= c1, c2 <= 4096"); return CMSVD_INVALID_ARG; }
    // X == Y (same buffer and leading dimension) selects the symmetric plan, which may use more chunks
    size_t a = gram_partials_size(c1, c2, n, ctx->sm_count, 0);
    size_t b = c1 == c2 ? gram_partials_size(c1, c2, n, ctx->sm_count, 1) : 0;
    *bytes = sizeof(double) * (a > b ? a : b) + 256;
    return CMSVD_OK;
}

int cmsvd_gram(cmsvd_context* ctx, int64_t n, int32_t c1, int32_t c2, const double* X, int64_t ldx, const double* Y,
               int64_t ldy, double* G, void* workspace, size_t ws_bytes) {
    size_t need = 0;
    CM_TRY(cmsvd_gram_workspace_size(ctx, n, c1, c2, &need));
    if (!X || !Y || !G || !workspace) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    if (ldx < c1 || ldy < c2) { set_error("need ldx >= c1 and ldy >= c2"); return CMSVD_INVALID_ARG; }
    if (ws_bytes < need) { set_error("workspace %zu < %zu bytes", ws_bytes, need); return CMSVD_WORKSPACE_TOO_SMALL; }
    Session se;
    CM_TRY(se.open(ctx));
    CM_TRY(gram(X, ldx, c1, Y, ldy, c2, n, G, (double*)workspace, (ws_bytes - 256) / sizeof(double), ctx->sm_count,
                ctx->s));
    return se.close();
}

int cmsvd_gemm(cmsvd_context* ctx, int64_t n, int32_t c1, int32_t c2, const double* X, int64_t ldx, const double* W,
               int64_t ldw, double* Z, int64_t ldz) {
    if (!ctx || !X || !W || !Z) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    if (n < 1 || c1 < 1 || c2 < 1 || c1 > 4096 || c2 > 4096 || ldx < c1 || ldw < c2 || ldz < c2) {
        set_error("need n >= 1, 1 <= c1, c2 <= 4096, ldx >= c1, ldw >= c2, ldz >= c2");
        return CMSVD_INVALID_ARG;
    }
    Session se;
    CM_TRY(se.open(ctx));
    CM_TRY(gemm_nn(X, ldx, W, ldw, Z, ldz, n, c1, c2, ctx->s, 0));
    return se.close();
}

int cmsvd_workspace_size(const cmsvd_matrix* A, const cmsvd_params* p, size_t* bytes) {
    if (!A || !p || !bytes) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    Arena ws;
    Plan pl;
    plan_persistent(ws, A, p, pl, true);
    *bytes = pl.persistent + scratch_size(A, p, true) + 1024;
    return CMSVD_OK;
}

int cmsvd_moments(cmsvd_matrix* A, double a, double b, const cmsvd_params* p, const double* V_in, double* S_out,
                  void* workspace, size_t ws_bytes, cmsvd_stats* stats) {
    CM_TRY(check_params(A, a, b, p));
    if (!V_in || !S_out || !workspace) { set_error("NULL V_in, S_out or workspace"); return CMSVD_INVALID_ARG; }
    size_t need = 0;
    CM_TRY(cmsvd_workspace_size(A, p, &need));
    if (ws_bytes < need) { set_error("workspace %zu < %zu bytes", ws_bytes, need); return CMSVD_WORKSPACE_TOO_SMALL; }
    cmsvd_context* ctx = A->ctx;
    Session se;
    CM_TRY(se.open(ctx));
    prof_reset(p->profile != 0);
    Arena ws;
    ws.base = (char*)workspace;
    ws.cap = ws_bytes;
    Plan pl;
    plan_persistent(ws, A, p, pl, false);
    cmsvd_stats st{};
    int status = run_moments(A, a, b, p, V_in, pl, ws, &st);
    if (status != CMSVD_OK && status != CMSVD_NOT_CONVERGED) return status;
    const size_t bytes = sizeof(double) * A->A.n * p->L * (p->M + 1);
    CM_CUDA(cudaMemcpyAsync(S_out, pl.S, bytes, cudaMemcpyDeviceToDevice, ctx->s));
    CM_CUDA(cudaStreamSynchronize(ctx->s));
    prof_collect(&st);
    if (stats) *stats = st;
    CM_TRY(se.close());
    return status;
}

int cmsvd_solve_interval(cmsvd_matrix* A, double a, double b, const cmsvd_params* p, const double* V_in, void* workspace,
                         size_t ws_bytes, cmsvd_result** out) {
    if (!out) { set_error("NULL out"); return CMSVD_INVALID_ARG; }
    *out = nullptr;
    CM_TRY(check_params(A, a, b, p));
    if (!V_in || !workspace) { set_error("NULL V_in or workspace"); return CMSVD_INVALID_ARG; }
    size_t need = 0;
    CM_TRY(cmsvd_workspace_size(A, p, &need));
    if (ws_bytes < need) { set_error("workspace %zu < %zu bytes", ws_bytes, need); return CMSVD_WORKSPACE_TOO_SMALL; }
    cmsvd_context* ctx = A->ctx;
    Session se;
    CM_TRY(se.open(ctx));
    Events ev;
    CM_TRY(ev.make());
    prof_reset(p->profile != 0);
    Arena ws;
    ws.base = (char*)workspace;
    ws.cap = ws_bytes;
    Plan pl;
    plan_persistent(ws, A, p, pl, true);
    cmsvd_stats st{};
    double normA = 0.0;
    CM_TRY(ensure_norm(A, p, ws, &normA));
    st.norm_A = normA;
    CM_CUDA(cudaEventRecord(ev.e[0], ctx->s));
    int status = run_moments(A, a, b, p, V_in, pl, ws, &st);
    if (status != CMSVD_OK && status != CMSVD_NOT_CONVERGED) return status;
    CM_CUDA(cudaEventRecord(ev.e[4], ctx->s));
    const int c = p->L * p->M;
    CM_TRY(rayleigh_ritz(A, pl.S, (int64_t)p->L * (p->M + 1), c, a, b, p, normA, ws, pl.out, &st, ev.e));
    CM_CUDA(cudaStreamSynchronize(ctx->s));
    prof_collect(&st);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev.e[0], ev.e[4]) == cudaSuccess) st.ms_solve = ms;
    if (cudaEventElapsedTime(&ms, ev.e[4], ev.e[1]) == cudaSuccess) st.ms_truncate = ms;
    if (cudaEventElapsedTime(&ms, ev.e[1], ev.e[2]) == cudaSuccess) st.ms_qr = ms;
    if (cudaEventElapsedTime(&ms, ev.e[2], ev.e[3]) == cudaSuccess) st.ms_ritz = ms;
    cudaGetLastError();
    cmsvd_result* r = new (std::nothrow) cmsvd_result();
    if (!r) { set_error("host allocation failed"); return CMSVD_OUT_OF_MEMORY; }
    r->m = A->A.m;
    r->n = A->A.n;
    r->t = st.found;
    r->ctx = ctx;
    r->sigma = pl.out.sigma;
    r->U = pl.out.U;
    r->V = pl.out.V;
    r->res_u = pl.out.res_u;
    r->res_v = pl.out.res_v;
    r->tau = pl.out.tau;
    r->res_est = p->estimate ? pl.out.res_est : nullptr;
    if (r->t > 0) {
        double* h = (double*)malloc(sizeof(double) * 2 * r->t);
        if (h) {
            cudaMemcpy(h, r->res_u, sizeof(double) * r->t, cudaMemcpyDeviceToHost);
            cudaMemcpy(h + r->t, r->res_v, sizeof(double) * r->t, cudaMemcpyDeviceToHost);
            for (int64_t i = 0; i < r->t; ++i) {
                st.max_res_u = fmax(st.max_res_u, h[i]);
                st.max_res_v = fmax(st.max_res_v, h[r->t + i]);
            }
            free(h);
        }
    }
    r->stats = st;
    *out = r;
    CM_TRY(se.close());
    if (status == CMSVD_OK && st.rank >= c) status = CMSVD_SUBSPACE_SATURATED;
    return status;
}

int cmsvd_result_count(const cmsvd_result* r, int64_t* t) {
    if (!r || !t) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    *t = r->t;
    return CMSVD_OK;
}

int cmsvd_result_copy(const cmsvd_result* r, double* sigma, double* U, double* V, double* res_u, double* res_v, double* tau) {
    if (!r) { set_error("NULL result"); return CMSVD_INVALID_ARG; }
    if (r->t == 0) return CMSVD_OK;
    cudaStream_t s = r->ctx->s;
    const size_t t = (size_t)r->t;
    if (sigma) CM_CUDA(cudaMemcpyAsync(sigma, r->sigma, sizeof(double) * t, cudaMemcpyDefault, s));
    if (U) CM_CUDA(cudaMemcpyAsync(U, r->U, sizeof(double) * t * r->m, cudaMemcpyDefault, s));
    if (V) CM_CUDA(cudaMemcpyAsync(V, r->V, sizeof(double) * t * r->n, cudaMemcpyDefault, s));
    if (res_u) CM_CUDA(cudaMemcpyAsync(res_u, r->res_u, sizeof(double) * t, cudaMemcpyDefault, s));
    if (res_v) CM_CUDA(cudaMemcpyAsync(res_v, r->res_v, sizeof(double) * t, cudaMemcpyDefault, s));
    if (tau) CM_CUDA(cudaMemcpyAsync(tau, r->tau, sizeof(double) * t, cudaMemcpyDefault, s));
    CM_CUDA(cudaStreamSynchronize(s));
    return CMSVD_OK;
}

int cmsvd_result_copy_estimate(const cmsvd_result* r, double* res_est) {
    if (!r || !res_est) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    if (!r->res_est) { set_error("the solve ran without the residual estimate (estimate = 0)"); return CMSVD_NOT_SUPPORTED; }
    if (r->t == 0) return CMSVD_OK;
    CM_CUDA(cudaMemcpyAsync(res_est, r->res_est, sizeof(double) * (size_t)r->t, cudaMemcpyDefault, r->ctx->s));
    CM_CUDA(cudaStreamSynchronize(r->ctx->s));
    return CMSVD_OK;
}

int cmsvd_result_stats(const cmsvd_result* r, cmsvd_stats* stats) {
    if (!r || !stats) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    *stats = r->stats;
    return CMSVD_OK;
}

int cmsvd_result_destroy(cmsvd_result* r) {
    delete r;
    return CMSVD_OK;
}

}  // extern "C"
