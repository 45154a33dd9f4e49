// Serving loop with continuous batching: interval-SVD requests on resident matrices are
// queued and admitted, in arrival order, as soon as a slot is free and their workspace fits
// in what remains of the HBM budget. Every slot is one context (its own streams) driven by
// its own host thread, so the work of admitted requests overlaps on the GPU while later
// requests wait. A request's inputs (V_in) come from host memory and its result is copied
// back to host memory when it completes; its workspace is taken from the stream-ordered
// allocator for the length of the solve. Every solve is the same computation as a single
// cmsvd_solve_interval call, so a result does not depend on the requests it ran beside.
#include "internal.cuh"
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct SrvMatrix {
    cmsvd_matrix* base = nullptr;               // owns the device data (made on the upload context)
    std::vector<cmsvd_matrix*> views;           // one shallow copy per slot, bound to its context
    size_t bytes = 0;
};

struct SrvReq {
    int64_t ticket = 0;
    int mid = 0;
    double a = 0.0, b = 0.0;
    cmsvd_params p{};
    std::vector<double> vin;
    size_t ws = 0;
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
    int status = CMSVD_OK;
    std::string err;
    int64_t t = 0, m = 0, n = 0;
    std::vector<double> sigma, U, V, ru, rv, tau;
    cmsvd_stats st{};
};

bool acceptable(int st) { return st == CMSVD_OK || st == CMSVD_NOT_CONVERGED || st == CMSVD_SUBSPACE_SATURATED; }

size_t csr_bytes(const cmsvd::Csr& A) {
    return sizeof(int64_t) * (A.m + 1) + (sizeof(int32_t) + sizeof(double)) * A.nnz + (A.vals_f ? sizeof(float) * A.nnz : 0) +
           (A.vals_lo ? sizeof(float) * A.nnz : 0) + (A.vals_h ? sizeof(uint16_t) * A.nnz : 0) + sizeof(int32_t) * A.m;
}

}  // namespace

struct cmsvd_server {
    int device = 0;
    int slots = 0;
    size_t budget = 0, in_use = 0;
    std::vector<cudaStream_t> streams;          // per slot: the stream its requests' copies run on
    std::vector<cmsvd_context*> ctx;
    cudaStream_t ustream = nullptr;             // uploads of new matrices, apart from the slots,
    cmsvd_context* uctx = nullptr;              // so that they never share a context with a solve
    std::vector<SrvMatrix> mats;
    std::mutex mu;                              // queue, requests, matrix table, budget
    std::mutex umu;                             // uploads (the upload context)
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<SrvReq>> queue;
    std::map<int64_t, std::shared_ptr<SrvReq>> reqs;
    int64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

void process(cmsvd_server* S, int slot, SrvReq& r) {
    using namespace cmsvd;
    cudaSetDevice(S->device);
    cudaStream_t s = S->streams[slot];
    cmsvd_matrix* A = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);   // mats may grow while requests run
        A = S->mats[r.mid].views[slot];
    }
    const size_t vbytes = sizeof(double) * r.vin.size();
    void* ws = nullptr;
    double* vin_d = nullptr;
    if (cudaMallocAsync(&ws, r.ws, s) != cudaSuccess || cudaMallocAsync((void**)&vin_d, vbytes, s) != cudaSuccess) {
        cudaGetLastError();
        r.status = CMSVD_OUT_OF_MEMORY;
        r.err = "stream-ordered allocation of the workspace failed";
    } else if (cudaMemcpyAsync(vin_d, r.vin.data(), vbytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        r.status = CMSVD_CUDA_ERROR;
        r.err = "copy of V_in failed";
    } else {
        cmsvd_result* res = nullptr;
        r.status = cmsvd_solve_interval(A, r.a, r.b, &r.p, vin_d, ws, r.ws, &res);
        if (!acceptable(r.status)) r.err = cmsvd_last_error();
        if (res) {
            try {
                r.t = res->t;
                r.m = res->m;
                r.n = res->n;
                r.sigma.resize(r.t);
                r.U.resize((size_t)r.t * r.m);
                r.V.resize((size_t)r.t * r.n);
                r.ru.resize(r.t);
                r.rv.resize(r.t);
                r.tau.resize(r.t);
                cmsvd_result_copy(res, r.sigma.data(), r.U.data(), r.V.data(), r.ru.data(), r.rv.data(), r.tau.data());
                cmsvd_result_stats(res, &r.st);
            } catch (...) {
                r.t = 0;
                r.sigma.clear(), r.U.clear(), r.V.clear(), r.ru.clear(), r.rv.clear(), r.tau.clear();
                r.status = CMSVD_OUT_OF_MEMORY;
                r.err = "host allocation of the result failed";
            }
            cmsvd_result_destroy(res);
        }
    }
    if (vin_d) cudaFreeAsync(vin_d, s);
    if (ws) cudaFreeAsync(ws, s);
    cudaStreamSynchronize(s);
}

void worker(cmsvd_server* S, int slot) {
    cudaSetDevice(S->device);
    for (;;) {
        std::shared_ptr<SrvReq> r;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                return S->stop || (!S->queue.empty() && S->in_use + S->queue.front()->ws <= S->budget);
            });
            if (S->stop) return;
            r = S->queue.front();
            S->queue.pop_front();
            S->in_use += r->ws;
            r->t_start = Clock::now();
        }
        process(S, slot, *r);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->in_use -= r->ws;
            r->t_done = Clock::now();
            r->done = true;
        }
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

extern "C" {

int cmsvd_server_create(int slots, size_t hbm_budget, cmsvd_server** out) {
    using namespace cmsvd;
    if (!out || slots < 1 || slots > 64) { set_error("slots must be in [1, 64] and out non-NULL"); return CMSVD_INVALID_ARG; }
    *out = nullptr;
    int device = 0;
    size_t free_b = 0, total_b = 0;
    CM_CUDA(cudaGetDevice(&device));
    CM_CUDA(cudaMemGetInfo(&free_b, &total_b));
    cmsvd_server* S = new (std::nothrow) cmsvd_server();
    if (!S) { set_error("host allocation failed"); return CMSVD_OUT_OF_MEMORY; }
    S->device = device;
    S->budget = hbm_budget ? hbm_budget : (size_t)(0.8 * (double)free_b);
    {
        // keep freed workspaces in the stream-ordered pool (up to the budget) instead of
        // returning them to the driver at every synchronization
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = S->budget;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    }
    S->slots = slots;
    for (int i = 0; i < slots; ++i) {
        cudaStream_t st = nullptr;
        cmsvd_context* c = nullptr;
        int e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess ? cmsvd_context_create(st, &c) : CMSVD_CUDA_ERROR;
        if (e != CMSVD_OK) {
            if (st) cudaStreamDestroy(st);
            cmsvd_server_destroy(S);
            if (e == CMSVD_CUDA_ERROR) set_error("stream or context creation failed");
            return e;
        }
        S->streams.push_back(st);
        S->ctx.push_back(c);
    }
    {
        int e = cudaStreamCreateWithFlags(&S->ustream, cudaStreamNonBlocking) == cudaSuccess
                    ? cmsvd_context_create(S->ustream, &S->uctx) : CMSVD_CUDA_ERROR;
        if (e != CMSVD_OK) {
            cmsvd_server_destroy(S);
            if (e == CMSVD_CUDA_ERROR) set_error("stream or context creation failed");
            return e;
        }
    }
    try {
        for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker, S, i);
    } catch (...) {
        cmsvd_server_destroy(S);   // joins the workers already started
        set_error("could not start the worker threads");
        return CMSVD_OUT_OF_MEMORY;
    }
    *out = S;
    return CMSVD_OK;
}

int cmsvd_server_destroy(cmsvd_server* S) {
    if (!S) return CMSVD_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    for (auto& m : S->mats) {
        for (auto* v : m.views) delete v;      // shallow copies: the device data belongs to base
        cmsvd_csr_destroy(m.base);
    }
    for (auto* c : S->ctx) cmsvd_context_destroy(c);
    for (auto st : S->streams) cudaStreamDestroy(st);
    if (S->uctx) cmsvd_context_destroy(S->uctx);
    if (S->ustream) cudaStreamDestroy(S->ustream);
    delete S;
    return CMSVD_OK;
}

int cmsvd_server_add_matrix(cmsvd_server* S, int64_t m, int64_t n, int64_t nnz, const int64_t* rowptr,
                            const int32_t* colidx, const double* vals, int vals_on_device, int32_t storage, int* id) {
    using namespace cmsvd;
    if (!S || !id) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    cmsvd_matrix* base = nullptr;
    std::lock_guard<std::mutex> ulk(S->umu);   // one upload at a time on the upload context
    CM_TRY(cmsvd_csr_create(S->uctx, m, n, nnz, rowptr, colidx, vals, vals_on_device, storage, &base));
    // build what solves would otherwise create lazily, so that the per-slot views only read it
    int st = components_build(base);
    if (st == CMSVD_OK) st = csr_make_fp32(base);
    // the slots' streams read these arrays without waiting on the upload stream
    if (st == CMSVD_OK && cudaStreamSynchronize(S->uctx->s) != cudaSuccess) {
        set_error("upload of the matrix failed");
        st = CMSVD_CUDA_ERROR;
    }
    if (st != CMSVD_OK) { cmsvd_csr_destroy(base); return st; }
    SrvMatrix sm;
    sm.base = base;
    sm.bytes = csr_bytes(base->A) + csr_bytes(base->At);
    for (int i = 0; i < S->slots; ++i) {
        cmsvd_matrix* v = new (std::nothrow) cmsvd_matrix(*base);
        if (!v) {
            for (auto* x : sm.views) delete x;
            cmsvd_csr_destroy(base);
            set_error("host allocation failed");
            return CMSVD_OUT_OF_MEMORY;
        }
        v->ctx = S->ctx[i];
        sm.views.push_back(v);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    // a queued request was admitted against the matrices resident at its submission; the new
    // matrix must still leave it room, or the queue would stall behind it for good
    size_t resident = 0, queued = 0;
    for (auto& x : S->mats) resident += x.bytes;
    for (auto& q : S->queue) queued = std::max(queued, q->ws);
    if (S->in_use + sm.bytes > S->budget || resident + sm.bytes + queued > S->budget) {
        for (auto* x : sm.views) delete x;
        cmsvd_csr_destroy(base);
        set_error("matrix of %zu bytes exceeds what the HBM budget leaves beside the resident matrices and queued requests",
                  sm.bytes);
        return CMSVD_OUT_OF_MEMORY;
    }
    S->in_use += sm.bytes;   // resident matrices stay counted in in_use
    *id = (int)S->mats.size();
    S->mats.push_back(sm);
    return CMSVD_OK;
}

int cmsvd_server_submit(cmsvd_server* S, int id, double a, double b, const cmsvd_params* p, const double* V_in_host,
                        int64_t* ticket) {
    using namespace cmsvd;
    if (!S || !p || !V_in_host || !ticket) { set_error("NULL argument"); return CMSVD_INVALID_ARG; }
    cmsvd_matrix* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (id < 0 || id >= (int)S->mats.size()) { set_error("unknown matrix id %d", id); return CMSVD_INVALID_ARG; }
        base = S->mats[id].base;
    }
    size_t ws = 0;
    CM_TRY(cmsvd_workspace_size(base, p, &ws));
    if (p->L < 1 || p->L > 128) { set_error("L must be in [1, 128]"); return CMSVD_INVALID_ARG; }
    std::shared_ptr<SrvReq> r;
    try {
        r = std::make_shared<SrvReq>();
        r->vin.assign(V_in_host, V_in_host + (size_t)base->A.n * p->L);
    } catch (...) {
        set_error("host allocation failed");
        return CMSVD_OUT_OF_MEMORY;
    }
    r->mid = id;
    r->a = a;
    r->b = b;
    r->p = *p;
    r->ws = ws + sizeof(double) * r->vin.size();
    std::lock_guard<std::mutex> lk(S->mu);
    size_t resident = 0;
    for (auto& m : S->mats) resident += m.bytes;
    if (r->ws + resident > S->budget) {
        set_error("request needs %zu bytes of workspace; the HBM budget leaves %zu", r->ws, S->budget - resident);
        return CMSVD_OUT_OF_MEMORY;
    }
    r->ticket = S->next_ticket++;
    r->t_submit = Clock::now();
    S->queue.push_back(r);
    S->reqs[r->ticket] = r;
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return CMSVD_OK;
}

int cmsvd_server_wait(cmsvd_server* S, int64_t ticket, int timeout_ms, int64_t* t, int* solve_status, double* latency_ms,
                      double* queue_ms) {
    using namespace cmsvd;
    if (!S) { set_error("NULL server"); return CMSVD_INVALID_ARG; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) { set_error("unknown ticket %lld", (long long)ticket); return CMSVD_INVALID_ARG; }
    std::shared_ptr<SrvReq> r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return CMSVD_PENDING;
    if (t) *t = r->t;
    if (solve_status) *solve_status = r->status;
    if (latency_ms) *latency_ms = ms_between(r->t_submit, r->t_done);
    if (queue_ms) *queue_ms = ms_between(r->t_submit, r->t_start);
    if (!acceptable(r->status)) set_error("%s", r->err.c_str());
    return CMSVD_OK;
}

int cmsvd_server_take(cmsvd_server* S, int64_t ticket, int64_t capacity, double* sigma, double* U, double* V,
                      double* res_u, double* res_v, double* tau, cmsvd_stats* stats) {
    using namespace cmsvd;
    if (!S) { set_error("NULL server"); return CMSVD_INVALID_ARG; }
    std::shared_ptr<SrvReq> r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) { set_error("unknown ticket %lld", (long long)ticket); return CMSVD_INVALID_ARG; }
        if (!it->second->done) { set_error("request %lld is still running", (long long)ticket); return CMSVD_PENDING; }
        if (capacity < it->second->t) {
            set_error("buffers hold %lld triplets, the request found %lld", (long long)capacity, (long long)it->second->t);
            return CMSVD_INVALID_ARG;
        }
        r = it->second;
        S->reqs.erase(it);
    }
    auto put = [](double* dst, const std::vector<double>& src) {
        if (dst && !src.empty()) memcpy(dst, src.data(), sizeof(double) * src.size());
    };
    put(sigma, r->sigma);
    put(U, r->U);
    put(V, r->V);
    put(res_u, r->ru);
    put(res_v, r->rv);
    put(tau, r->tau);
    if (stats) *stats = r->st;
    return CMSVD_OK;
}

}  // extern "C"
