// Launch-shape autotuner for batched linear steps.
//
// The step's work per PCG iteration is fixed by the method; what the hardware
// makes of it depends on the launch shape: on the cluster path the column tile
// width and the CTAs per cluster, on the graph path the rows each block owns on
// the finest and on the coarser multigrid depths (grid size against the 152 SMs),
// halo-fused multigrid kernels or not, and the cores (CUDA or tensor) and column
// tiles per block of the dense base solve.  mg_autotune times
// one batched step per candidate shape with CUDA events and keeps the fastest,
// by coordinate descent from the library's own choice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <vector>

#include "internal.h"

namespace {

// fixed pseudo-random start states in [-0.01, 0.01] (a counter-based integer hash)
__global__ void kt_fill(int64_t n, double* x) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint64_t h = (uint64_t)q * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    x[q] = 0.01 * (2.0 * (double)(h >> 11) * (1.0 / 9007199254740992.0) - 1.0);
}

struct Trial {
    int path, tile, cluster, rbs0, rbs1, tb, hf, bc;
};

}  // namespace

extern mg_status mg_guarded_call(mg_ctx* c, void (*fn)(void*), void* arg);

extern "C" mg_status mg_autotune(mg_ctx* c, int level, int64_t N, double T, int k, mg_solver_opts* opts,
                                 double* best_ms) {
    struct Args {
        mg_ctx* c;
        int level;
        int64_t N;
        double T;
        int k;
        mg_solver_opts* opts;
        double* best_ms;
    } a{c, level, N, T, k, opts, best_ms};
    return mg_guarded_call(
        c,
        [](void* p) {
            Args& A = *static_cast<Args*>(p);
            mg_ctx* c = A.c;
            if (!A.opts || A.level < 0 || A.level >= (int)c->meshes.size() || A.N <= 0 || !(A.T > 0.0) ||
                A.k <= 0 || A.k > 65536)
                mg_fail(MG_EINVAL, "mg_autotune: bad arguments");
            ctx_finalize(c);
            if (mesh_is_nonlinear(c, A.level)) mg_fail(MG_EINVAL, "mg_autotune: times linear steps only");
            const StepOp& op = ctx_step_op(c, A.level, A.T / (double)A.N);
            const double* wave = ctx_wave_table(c, A.N, A.T, 0);
            const int64_t n = c->meshes[A.level].n;
            DBuf xin, xout;
            xin.ensure((size_t)n * A.k * sizeof(double));
            xout.ensure((size_t)n * A.k * sizeof(double));
            cudaStream_t s = c->stream;
            kt_fill<<<(unsigned)((n * A.k + 255) / 256), 256, 0, s>>>(n * A.k, xin.as<double>());
            MG_CUDA(cudaGetLastError());
            PhiIO io;
            io.k = A.k;
            io.xprev = xin.as<double>();
            io.ld_prev = A.k;
            io.xout = xout.as<double>();
            io.ld_out = A.k;
            io.wave = wave;
            io.t0 = std::min<int64_t>(1, A.N);
            io.tstride = A.k > 1 && io.t0 + (int64_t)(A.k - 1) <= A.N ? 1 : 0;
            cudaEvent_t e0, e1;
            MG_CUDA(cudaEventCreate(&e0));
            MG_CUDA(cudaEventCreate(&e1));
            auto time_of = [&](const Trial& t) {
                mg_solver_opts so = *A.opts;
                so.path = t.path;
                so.tile = t.tile;
                so.cluster = t.cluster;
                so.rows_per_block = t.rbs0;
                so.coarse_rows_per_block = t.rbs1;
                so.base_tiles = t.tb;
                so.halo_fusion = t.hf;
                so.base_cores = t.bc;
                if (mg_trace_level() >= 3) {
                    std::fprintf(stderr,
                                 "[autotune] mesh %d k %d path %d tile %d cluster %d rbs %d/%d tiles %d halo %d base %d\n",
                                 A.level, A.k, t.path, t.tile, t.cluster, t.rbs0, t.rbs1, t.tb, t.hf, t.bc);
                    MG_CUDA(cudaStreamSynchronize(s));
                }
                phi_batch(c, op, io, so, nullptr);  // builds the plan, warms the caches
                if (mg_trace_level() >= 3) MG_CUDA(cudaStreamSynchronize(s));
                MG_CUDA(cudaEventRecord(e0, s));
                for (int r = 0; r < 3; ++r) phi_batch(c, op, io, so, nullptr);
                MG_CUDA(cudaEventRecord(e1, s));
                MG_CUDA(cudaEventSynchronize(e1));
                float ms = 0.0f;
                MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                return (double)ms / 3.0;
            };
            Trial best{};
            double best_t = std::numeric_limits<double>::infinity();
            auto consider = [&](const Trial& t) {
                const double ms = time_of(t);
                if (ms < best_t) {
                    best_t = ms;
                    best = t;
                }
            };
            try {
                if (A.k < 32) {  // latency-bound: cluster tile width and size, or the graph path
                    for (int tile : {1, 8, 16})
                        for (int cl : {8, 16}) consider({MG_PATH_CLUSTER, tile, cl, 0, 0, 0, 0, 0});
                }
                Trial gb{MG_PATH_GRAPH, 0, 0, 0, 0, 0, 0, 0};
                double gt = time_of(gb);
                for (int r0 : {128, 256, 512, 1024}) {
                    Trial t = gb;
                    t.rbs0 = r0;
                    const double ms = time_of(t);
                    if (ms < gt) gt = ms, gb = t;
                }
                for (int hf : {1, 2, 3}) {
                    Trial t = gb;
                    t.hf = hf;
                    const double ms = time_of(t);
                    if (ms < gt) gt = ms, gb = t;
                }
                for (int r1 : {32, 64, 128, 256}) {
                    Trial t = gb;
                    t.rbs1 = r1;
                    const double ms = time_of(t);
                    if (ms < gt) gt = ms, gb = t;
                }
                for (int bc : {MG_BASE_CUDA, MG_BASE_TENSOR}) {
                    Trial t = gb;
                    t.bc = bc;
                    const double ms = time_of(t);
                    if (ms < gt) gt = ms, gb = t;
                }
                for (int tb : {1, 2, 4}) {
                    Trial t = gb;
                    t.tb = tb;
                    const double ms = time_of(t);
                    if (ms < gt) gt = ms, gb = t;
                }
                if (gt < best_t) best_t = gt, best = gb;
            } catch (...) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                ctx_drop_plans(c);
                throw;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            ctx_drop_plans(c);  // the trial plans; the chosen one is rebuilt on first use
            A.opts->path = best.path;
            A.opts->tile = best.tile;
            A.opts->cluster = best.cluster;
            A.opts->rows_per_block = best.rbs0;
            A.opts->coarse_rows_per_block = best.rbs1;
            A.opts->base_tiles = best.tb;
            A.opts->halo_fusion = best.hf;
            A.opts->base_cores = best.bc;
            c->tuned[{A.level, tune_bucket(A.k)}] = {best.path, best.tile, best.cluster, best.rbs0, best.rbs1,
                                                     best.tb,   best.hf,   best.bc,      best_t};
            if (A.best_ms) *A.best_ms = best_t;
        },
        &a);
}

// ------------------------------------------------------------------ temporal coarsening plan
//
// Sec. 4.1 chooses a large first coarsening factor so that the second time grid
// has one point per processor, and a small factor on the coarser grids (2 in its
// worked example, 4 in the runs of Secs. 4.2 and 5).  On one GPU the
// counterpart of "one point per processor" is the batch width from which a
// batched step stops gaining throughput: the first factor makes the finest
// relaxation batches that wide.

extern "C" mg_status mg_choose_levels(const double* k_list, const double* ms_list, int nk, int64_t N, int max_levels,
                                      int coarse_m, int* levels_out, int* m_out) {
    if (!k_list || !ms_list || nk <= 0 || N < 2 || max_levels < 2 || max_levels > 8 || coarse_m < 0 ||
        coarse_m == 1 || !levels_out || !m_out)
        return MG_EINVAL;
    const int64_t cm = coarse_m ? coarse_m : 2;
    double best = 0.0;
    for (int i = 0; i < nk; ++i) {
        if (!(k_list[i] >= 1.0) || !(ms_list[i] > 0.0)) return MG_EINVAL;
        best = std::max(best, k_list[i] / ms_list[i]);
    }
    double kstar = 0.0;
    for (int i = 0; i < nk; ++i)
        if (k_list[i] / ms_list[i] >= 0.9 * best && (kstar == 0.0 || k_list[i] < kstar)) kstar = k_list[i];
    // first factor: the largest divisor of N with N / m0 >= kstar (at least 2)
    int64_t m0 = 0;
    for (int64_t m = std::min<int64_t>(N / 2, (int64_t)(N / std::max(1.0, kstar))); m >= 2; --m)
        if (N % m == 0 && (double)(N / m) >= kstar) {
            m0 = m;
            break;
        }
    if (!m0) return MG_EINVAL;
    int levels = 2;
    m_out[0] = (int)m0;
    int64_t Nl = N / m0;
    while (levels < max_levels && Nl % cm == 0 && Nl / cm >= 2) {
        m_out[levels - 1] = (int)cm;
        Nl /= cm;
        ++levels;
    }
    for (int l = levels - 1; l < 8; ++l) m_out[l] = 0;
    *levels_out = levels;
    return MG_OK;
}

extern "C" mg_status mg_plan_levels(mg_ctx* c, int fine_level, int coarse_level, int64_t N, double T, int max_levels,
                                    mg_opts* opts, double* iter_ms) {
    struct Args {
        mg_ctx* c;
        int fine, coarse;
        int64_t N;
        double T;
        int max_levels;
        mg_opts* opts;
        double* iter_ms;
    } a{c, fine_level, coarse_level, N, T, max_levels, opts, iter_ms};
    return mg_guarded_call(
        c,
        [](void* p) {
            Args& A = *static_cast<Args*>(p);
            mg_ctx* c = A.c;
            if (!A.opts || A.fine < 0 || A.fine >= (int)c->meshes.size() || A.coarse < 0 ||
                A.coarse >= (int)c->meshes.size() || A.N < 2 || !(A.T > 0.0))
                mg_fail(MG_EINVAL, "mg_plan_levels: bad arguments");
            ctx_finalize(c);
            if (mesh_is_nonlinear(c, A.fine)) mg_fail(MG_EINVAL, "mg_plan_levels: times linear steps only");
            // step time against batch width on the fine mesh (library shapes)
            std::vector<double> ks, ms;
            auto time_step = [&](int mesh, int64_t Nl, int k) {
                const StepOp& op = ctx_step_op(c, mesh, A.T / (double)Nl);
                const double* wave = ctx_wave_table(c, A.N, A.T, 0);
                const int64_t n = c->meshes[mesh].n;
                DBuf xin, xout;
                xin.ensure((size_t)n * k * sizeof(double));
                xout.ensure((size_t)n * k * sizeof(double));
                kt_fill<<<(unsigned)((n * k + 255) / 256), 256, 0, c->stream>>>(n * k, xin.as<double>());
                PhiIO io;
                io.k = k;
                io.xprev = xin.as<double>();
                io.ld_prev = k;
                io.xout = xout.as<double>();
                io.ld_out = k;
                io.wave = wave;
                io.t0 = 1;
                io.tstride = (k > 1 && 1 + (int64_t)(k - 1) * (A.N / Nl) <= A.N) ? A.N / Nl : 0;
                mg_solver_opts so = A.opts->solver;
                phi_batch(c, op, io, so, nullptr);
                cudaEvent_t e0, e1;
                MG_CUDA(cudaEventCreate(&e0));
                MG_CUDA(cudaEventCreate(&e1));
                MG_CUDA(cudaEventRecord(e0, c->stream));
                for (int r = 0; r < 2; ++r) phi_batch(c, op, io, so, nullptr);
                MG_CUDA(cudaEventRecord(e1, c->stream));
                MG_CUDA(cudaEventSynchronize(e1));
                float t = 0.0f;
                MG_CUDA(cudaEventElapsedTime(&t, e0, e1));
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return (double)t / 2.0;
            };
            for (int k = 16; k <= 1024 && k <= A.N / 2; k *= 2) {
                ks.push_back(k);
                ms.push_back(time_step(A.fine, A.N, k));
            }
            int levels = 0, m[8] = {};
            if (mg_choose_levels(ks.data(), ms.data(), (int)ks.size(), A.N, std::max(2, A.max_levels), 0, &levels, m) !=
                MG_OK)
                mg_fail(MG_EINVAL, "mg_plan_levels: N has no power-of-two coarsening");
            // candidate hierarchies: the heuristic's and fixed factors that divide N; each
            // runs a few MGRIT iterations, and the one with the least predicted time to
            // the tolerance is chosen (measured time per iteration x iterations predicted
            // from the measured residual reduction per iteration)
            std::vector<std::vector<int>> cands;
            cands.push_back(std::vector<int>(m, m + levels - 1));
            for (auto f : std::vector<std::vector<int>>{{16}, {16, 16}, {32, 16}, {8, 8, 8}}) {
                int64_t prod = 1;
                for (int v : f) prod *= v;
                if ((int)f.size() + 1 <= std::max(2, A.max_levels) && A.N % prod == 0 && A.N / prod >= 2 &&
                    f != cands[0])
                    cands.push_back(f);
            }
            const int probe_iters = 4;
            const double tol = A.opts->tol > 0.0 ? A.opts->tol : 1e-10;
            double best_t = std::numeric_limits<double>::infinity(), best_it_ms = 0.0;
            std::vector<int> best_m = cands[0];
            for (const auto& f : cands) {
                mg_opts o = *A.opts;
                o.levels = (int)f.size() + 1;
                for (int l = 0; l < 8; ++l) {
                    o.m[l] = l < (int)f.size() ? f[l] : 0;
                    o.space_level[l] = l == 0 ? A.fine : A.coarse;
                }
                std::vector<double> hist;
                double secs = 0.0;
                mgrit_probe(c, A.N, A.T, o, probe_iters, hist, secs);
                const double it_ms = 1e3 * secs / (double)std::max<size_t>(1, hist.size());
                // reduction per iteration after the first (the first carries the start-up transient)
                double rho = 1.0;
                if (hist.size() >= 3 && hist[1] > 0.0) {
                    const double last = hist.back();
                    rho = last > 0.0 ? std::pow(last / hist[1], 1.0 / (double)(hist.size() - 2)) : 0.0;
                }
                double iters = std::numeric_limits<double>::infinity();
                if (rho == rho && rho <= 0.0) iters = (double)hist.size();
                else if (rho == rho && rho < 1.0) iters = 1.0 + std::ceil(std::log(tol) / std::log(rho));
                const double t = iters * it_ms;
                if (mg_trace_level() >= 1)
                    std::fprintf(stderr, "[plan] levels %d m %d %d %d: %.3f ms/iteration, reduction %.3f, %.0f iterations\n",
                                 o.levels, o.m[0], o.m[1], o.m[2], it_ms, rho, iters);
                if (t < best_t) {
                    best_t = t;
                    best_it_ms = it_ms;
                    best_m = f;
                }
            }
            ctx_drop_plans(c);
            A.opts->levels = (int)best_m.size() + 1;
            for (int l = 0; l < 8; ++l) {
                A.opts->m[l] = l < (int)best_m.size() ? best_m[l] : 0;
                A.opts->space_level[l] = l == 0 ? A.fine : A.coarse;
            }
            if (A.iter_ms) *A.iter_ms = best_it_ms;
        },
        &a);
}
