// Many independent machine instances at once.
//
// An instance is one context (meshes, materials, PWM, its own CUDA stream) and
// one solve.  Small instances leave most of the GPU idle (their batched steps
// have few columns, their coarsest levels are sequential), so solving them one
// after another wastes the machine.  mg_batch_solve gives every instance a host
// worker thread that drives its context's stream; the instances' kernels and
// CUDA graphs then run concurrently on the GPU, each with its own work buffers.
//
// Uneven instances can need more device memory together than the GPU has (an
// MGRIT solve keeps about one and a half trajectories of work storage besides its
// output).  With a work budget the scheduler admits instances largest first while
// the estimated work buffers of the running ones fit it, and frees each
// instance's buffers when it ends, so that the peak stays within the budget while
// the small instances fill the GPU around the large ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "job_sched.h"

namespace {

mg_status solve_one(mg_ctx* c, int64_t N, double T, const double* a0, double* out, const mg_opts& o,
                    mg_stats* si) {
    mg_status st = o.levels <= 1 ? mg_sequential(c, o.space_level[0], N, T, a0, out, &o.solver, si)
                                 : mg_solve(c, N, T, a0, out, &o, si);
    // the instance is finished when its stream is
    if (cudaSetDevice(c->device) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
        if (st == MG_OK) st = MG_ECUDA;
    return st;
}

}  // namespace

extern "C" mg_status mg_batch_solve(mg_ctx* const* ctxs, int n, const int64_t* N, const double* T,
                                    const double* const* a0, double* const* out, const mg_opts* opts,
                                    int max_threads, int64_t work_budget, mg_status* status, mg_stats* stats) {
    if (n <= 0 || !ctxs || !N || !T || !a0 || !out || !opts || max_threads < 0 || work_budget < -1) return MG_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return MG_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return MG_EINVAL;  // a context serves one instance at a time
    }
    // admission bound and per-instance estimates
    size_t budget = 0;
    if (work_budget == -1) {
        size_t free_b = 0, total_b = 0;
        if (cudaSetDevice(ctxs[0]->device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess)
            return MG_ECUDA;
        budget = std::max<size_t>(1, free_b - free_b / 20);
    } else if (work_budget > 0) {
        budget = (size_t)work_budget;
    }
    std::vector<size_t> est(n, 0);
    if (budget)
        for (int i = 0; i < n; ++i) {
            int64_t b = 0;
            if (mg_solve_work_bytes(ctxs[i], N[i], &opts[i], &b) == MG_OK) est[i] = (size_t)b;
        }
    std::vector<int> st;
    const bool started = mgsched::run_jobs(
        n, est, budget, max_threads,
        [&](int i) {
            return (int)solve_one(ctxs[i], N[i], T[i], a0[i], out[i], opts[i], stats ? &stats[i] : nullptr);
        },
        [&](int i) { mg_release_work(ctxs[i]); }, st, (int)MG_ENOMEM);
    if (!started) return MG_ENOMEM;
    mg_status worst = MG_OK;
    for (int i = 0; i < n; ++i) {
        if (status) status[i] = (mg_status)st[i];
        if (st[i] != MG_OK && (worst == MG_OK || st[i] < worst)) worst = (mg_status)st[i];
    }
    return worst;
}
