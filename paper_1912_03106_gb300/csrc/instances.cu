// Many independent machine instances at once.
//
// An instance is one context (meshes, materials, PWM, its own CUDA stream) and
// one solve.  Small instances leave most of the GPU idle (their batched steps
// have few columns, their coarsest levels are sequential), so solving them one
// after another wastes the machine.  mg_batch_solve gives every instance a host
// worker thread that drives its context's stream; the instances' kernels and
// CUDA graphs then run concurrently on the GPU, each with its own work buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "internal.h"

extern "C" mg_status mg_batch_solve(mg_ctx* const* ctxs, int n, const int64_t* N, const double* T,
                                    const double* const* a0, double* const* out, const mg_opts* opts,
                                    int max_threads, mg_status* status, mg_stats* stats) {
    if (n <= 0 || !ctxs || !N || !T || !a0 || !out || !opts || max_threads < 0) return MG_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return MG_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return MG_EINVAL;  // a context serves one instance at a time
    }
    std::vector<mg_status> st(n, MG_OK);
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) {
            mg_stats* si = stats ? &stats[i] : nullptr;
            st[i] = opts[i].levels <= 1
                        ? mg_sequential(ctxs[i], opts[i].space_level[0], N[i], T[i], a0[i], out[i], &opts[i].solver, si)
                        : mg_solve(ctxs[i], N[i], T[i], a0[i], out[i], &opts[i], si);
            // the instance is finished when its stream is
            mg_ctx* c = ctxs[i];
            if (cudaSetDevice(c->device) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
                if (st[i] == MG_OK) st[i] = MG_ECUDA;
        }
    };
    const int nt = max_threads == 0 ? n : std::min(n, max_threads);
    std::vector<std::thread> pool;
    pool.reserve(nt);
    try {
        for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    } catch (...) {
        for (auto& th : pool) th.join();
        return MG_ENOMEM;
    }
    for (auto& th : pool) th.join();
    mg_status worst = MG_OK;
    for (int i = 0; i < n; ++i) {
        if (status) status[i] = st[i];
        if (st[i] != MG_OK && (worst == MG_OK || st[i] < worst)) worst = st[i];
    }
    return worst;
}
