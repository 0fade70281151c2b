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
#include <condition_variable>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "internal.h"

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
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    if (budget) {
        for (int i = 0; i < n; ++i) {
            int64_t b = 0;
            if (mg_solve_work_bytes(ctxs[i], N[i], &opts[i], &b) == MG_OK) est[i] = (size_t)b;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return est[a] > est[b]; });
    }
    std::vector<mg_status> st(n, MG_OK);
    std::vector<int> retry;
    std::mutex mu;
    std::condition_variable cv;
    size_t in_use = 0;
    int running = 0, next = 0;
    auto worker = [&]() {
        for (;;) {
            std::unique_lock<std::mutex> lk(mu);
            if (next >= n) return;
            const int i = order[next++];
            if (budget) cv.wait(lk, [&] { return running == 0 || in_use + est[i] <= budget; });
            in_use += est[i];
            ++running;
            lk.unlock();
            mg_stats* si = stats ? &stats[i] : nullptr;
            st[i] = solve_one(ctxs[i], N[i], T[i], a0[i], out[i], opts[i], si);
            if (budget) mg_release_work(ctxs[i]);
            lk.lock();
            in_use -= est[i];
            --running;
            if (budget && st[i] == MG_ENOMEM) retry.push_back(i);
            lk.unlock();
            cv.notify_all();
        }
    };
    const int nt = max_threads == 0 ? n : std::min(n, max_threads);
    std::vector<std::thread> pool;
    pool.reserve(nt);
    try {
        for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(mu);
            next = n;  // no further instance starts
        }
        cv.notify_all();
        for (auto& th : pool) th.join();
        return MG_ENOMEM;
    }
    for (auto& th : pool) th.join();
    // instances that ran out of memory next to others, now alone
    for (int i : retry) {
        mg_stats* si = stats ? &stats[i] : nullptr;
        st[i] = solve_one(ctxs[i], N[i], T[i], a0[i], out[i], opts[i], si);
        mg_release_work(ctxs[i]);
    }
    mg_status worst = MG_OK;
    for (int i = 0; i < n; ++i) {
        if (status) status[i] = st[i];
        if (st[i] != MG_OK && (worst == MG_OK || st[i] < worst)) worst = st[i];
    }
    return worst;
}
