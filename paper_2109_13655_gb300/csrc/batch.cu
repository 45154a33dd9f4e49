// Batched solves: many independent interval-SVD problems at once. Problems whose matrices
// share a context run one after another on that context's stream; distinct contexts run
// concurrently, each driven by its own host thread, so the small kernels and host
// round trips of one solve overlap with the work of the others on the GPU. Every solve is
// the same computation as a single cmsvd_solve_interval call (deterministic kernels, no
// shared state between contexts), so its result does not depend on the batch it ran in.
#include "internal.cuh"
#include <map>
#include <string>
#include <thread>
#include <vector>

namespace {

bool acceptable(int st) { return st == CMSVD_OK || st == CMSVD_NOT_CONVERGED || st == CMSVD_SUBSPACE_SATURATED; }

}  // namespace

extern "C" int cmsvd_solve_batch(int count, cmsvd_matrix* const* A, const double* a, const double* b,
                                 const cmsvd_params* p, const double* const* V_in, void* const* workspace,
                                 const size_t* ws_bytes, cmsvd_result** out, int* status) {
    using namespace cmsvd;
    if (count < 0 || (count > 0 && (!A || !a || !b || !p || !V_in || !workspace || !ws_bytes || !out || !status))) {
        set_error("NULL argument or negative count");
        return CMSVD_INVALID_ARG;
    }
    std::map<cmsvd_context*, std::vector<int>> groups;
    for (int i = 0; i < count; ++i) {
        out[i] = nullptr;
        status[i] = CMSVD_INVALID_ARG;
        if (!A[i] || !A[i]->ctx) { set_error("problem %d: NULL matrix", i); return CMSVD_INVALID_ARG; }
        groups[A[i]->ctx].push_back(i);
    }
    std::vector<std::vector<int>> work;
    for (auto& g : groups) work.push_back(g.second);
    std::vector<std::string> errs(count);   // per problem: the error text of its thread
    auto run = [&](size_t w) {
        for (int i : work[w]) {
            status[i] = cmsvd_solve_interval(A[i], a[i], b[i], p + i, V_in[i], workspace[i], ws_bytes[i], out + i);
            if (!acceptable(status[i])) errs[i] = cmsvd_last_error();
        }
    };
    std::vector<std::thread> threads;
    for (size_t w = 1; w < work.size(); ++w) {
        try {
            threads.emplace_back(run, w);
        } catch (...) {
            run(w);   // no thread to be had: run this context's problems here
        }
    }
    if (!work.empty()) run(0);
    for (auto& t : threads) t.join();
    for (int i = 0; i < count; ++i) {
        if (!acceptable(status[i])) {
            set_error("problem %d: %s", i, errs[i].c_str());
            return status[i];
        }
    }
    return CMSVD_OK;
}
