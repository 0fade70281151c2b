// Batched backward-Euler step solves for large batches: one high-occupancy kernel
// per phase over all column tiles, the PCG loop inside one CUDA graph.
//
// Same mathematics as the cluster-resident kernel (pcg.cu): per column the step
// of Eq. discrete_system solved by PCG with one FP32 multigrid V-cycle as the
// preconditioner, FP64 form or FP32 inner iterations inside FP64 refinement.
// Here every phase is its own kernel over a (tile, 256-row block) grid with
// float4 / double2 lanes and a small register footprint, so all SMs run many
// warps and the memory system, not latency, sets the pace.  Per-column dot
// products are reduced in two deterministic stages: each block writes its
// per-column partial, and a one-block scalar kernel adds the partials of all
// row blocks in a fixed order and updates the per-column PCG scalars.  The
// iteration loop is a graph conditional WHILE node whose condition the
// convergence kernel sets on the device, so one graph launch runs a whole batched
// step without host round trips.  The per-call arguments (pointers, time indices,
// tolerances) are read from a small device struct, so the instantiated graph is
// reused by every call with the same operator and tile count.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
// Phases are separate kernels here, so L1-cached loads of work vectors are coherent.
#define MG_L1 1
#include "vec.cuh"

namespace {

using namespace mgv;

constexpr int G = 16;     // columns per tile
constexpr int NTB = 256;  // threads per block
// rows per block: MG_RBS0 on the finest depth (MG_RBS0_LARGE above 8,192 rows),
// MG_RBS1 on coarser depths, so that a 4,512-row depth still spreads over all SMs
#ifndef MG_RBS0
#define MG_RBS0 256
#endif
#ifndef MG_RBS0_LARGE
#define MG_RBS0_LARGE 512
#endif
#ifndef MG_RBS1
#define MG_RBS1 64
#endif
// Programmatic dependent launch between consecutive phase kernels (MG_PDL = 1):
// each kernel waits for its predecessor's completion (griddepcontrol.wait) before
// touching its outputs and lets its own successor be scheduled as soon as all of
// its blocks run (griddepcontrol.launch_dependents).  Measured on GB300 it slows
// the 18,240 x 256 step (12.2 against 11.4 ms): the early successor blocks take
// resources from the running phase.  Off by default.
#ifndef MG_PDL
#define MG_PDL 0
#endif
__device__ __forceinline__ void phase_begin() {
#if MG_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// minimum resident blocks per SM for the FP32 multigrid kernels (caps registers)
#ifndef MG_MINB_F
#define MG_MINB_F 5
#endif

struct CallArgs {
    const double* xprev;
    int64_t ld_prev;
    const double* g;
    int64_t ld_g;
    const double* guess;
    int64_t ld_guess;
    double* xout;
    int64_t ld_out;
    const double* wave;
    int64_t t0, tstride;
    int k;
    double tol2;        // FP64 form: cg_tol^2; FP32+refine: refine_tol^2
    double inner_tol2;  // FP32+refine: reduction^2 of the FP32 residual that triggers an FP64 update
    // rounding floor of the FP64 residual b - L x: a column whose computed residual
    // satisfies ||r||^2 <= fl_acc2 * S^2, S = || |b| + |L| |x| ||, is a solution to
    // working precision (its initial guess is kept, refinement stops); the PCG
    // iteration stops at fl_stop2 * S^2 (0: no floor)
    double fl_stop2, fl_acc2;
    int max_it;
    int max_refine;
};

struct Depth {
    int n, W, nrb, rbs;  // rows, ELL width, row blocks per tile, rows per block
    const int32_t* col;
    const double* L64;
    const double* M64;
    const float* L32;
    const float* Llo32;  // shared operators: L64 - L32 in FP32 (double-float operator products)
    const float *M32, *Mlo32;  // shared operators: M64 as two FP32 parts
    const float* LD32;
    const float* dinv32;
    const int32_t* par;  // transfer to the next coarser depth
    const float* pw;
    int rt_W;
    const int32_t* rt_col;
    const float* rt_w;
    float *x, *sa, *sb, *y, *r;
    // per column tile: 0 once all of its columns have stopped iterating; the PCG and
    // multigrid kernels then skip the tile (its vectors and partials stay as they are)
    const int* tact;
    // halo-fused kernels (kb_smooth2, kb_prolong_res): columns and rows per block,
    // the operator's bandwidth max |i - j|, the row blocks per column group and
    // whether the sweeps' input is staged in shared memory too; f_cw = 0: one
    // sweep and one transfer per launch
    int f_cw, f_R, f_H, f_nrb, f_stage;
};

struct Cols {
    double *bb, *gam, *beta, *alpha, *ref, *prev, *ss;  // ss: S^2 of the rounding floor
    int *act, *outer, *iters;
    int* bad;  // a non-finite residual or right-hand side was seen (reported as MG_ENONFINITE)
    int *upd, *nup, *stall;  // FP32+refine: FP64 update due, updates done, updates without progress
    int* lastu;              // FP32+refine: the column's iteration count at its last FP64 update
    int* tact;               // per tile: any column still iterating (see Depth::tact)
    int* ctr;  // [0] iterations of the current PCG, [1] refinement sweep
};

__device__ __forceinline__ void tile_rb(int nrb, int& t, int& rb) {
    t = blockIdx.x / nrb;
    rb = blockIdx.x - t * nrb;
}

// false once every column of tile t has stopped iterating (block-uniform)
__device__ __forceinline__ bool tile_on(const int* tact, int t) { return !tact || __ldg(tact + t) != 0; }

// Per-block, per-column sum of the thread's V column partials into part[blockIdx.x * G + c].
template <int V>
__device__ __forceinline__ void block_partial(double (&v)[V], double* part) {
    constexpr int TPR = G / V;
    __shared__ double red[NTB / 32][G];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < V; ++e) {
#pragma unroll
        for (int off = TPR; off < 32; off <<= 1) v[e] += __shfl_xor_sync(0xffffffffu, v[e], off);
    }
    if (lane < TPR) {
#pragma unroll
        for (int e = 0; e < V; ++e) red[warp][lane * V + e] = v[e];
    }
    __syncthreads();
    if (threadIdx.x < G) {
        double s = 0.0;
        for (int w = 0; w < NTB / 32; ++w) s += red[w][threadIdx.x];
        part[(size_t)blockIdx.x * G + threadIdx.x] = s;
    }
}

// sum over the row blocks of column gc (fixed order)
__device__ __forceinline__ double col_total(const double* part, int nrb, int gc) {
    const int t = gc / G, l = gc % G;
    double s = 0.0;
    for (int rb = 0; rb < nrb; ++rb) s += part[((size_t)t * nrb + rb) * G + l];
    return s;
}


template <class T>
__device__ __forceinline__ T* tv(T* base, int n, int t) { return base + (size_t)t * n * G; }

// Double-float operator products (DfAcc) serve the FP64 form's steps whose
// tolerance leaves room for their accuracy (about 2^-46 of sum |L_ij z_j| against
// FP64's 2^-50): cg_tol >= 1e-8, where the resulting drift of the recursive
// residual stays orders of magnitude below the stop test.  The FP64 form launches
// both variants of kb_pcg_a; the one that this call's tolerance (read on the
// device) does not select returns at once, and each keeps its own register budget.
// kb_init's products have FP64 operands on both sides: kb_split first writes
// x_prev and the guess as two FP32 parts each, once per step (splitting each value
// at every one of its ~7 gathers measured slower than the FP64 pipe: 246 against
// 218 us at 18,240 x 256), and kb_init's double-float variant gathers those parts.
constexpr double kDfTol2 = 1e-16;
__device__ __forceinline__ bool use_df(const Depth& D, const CallArgs* ca) {
    return D.Llo32 && ca->tol2 >= kDfTol2;
}
__device__ __forceinline__ bool use_df_init(const Depth& D, const CallArgs* ca) {
    return use_df(D, ca) && D.M32 && !ca->g;
}

// x_prev and the guess (FP64, the caller's layout) as two FP32 parts each,
// tile-major, for kb_init's double-float variant; returns at once when that
// variant does not run this call.  The guess parts are zero without a guess.
__global__ void __launch_bounds__(NTB) kb_split(Depth D, const CallArgs* __restrict__ ca, float* ph, float* pl,
                                                float* gh, float* gl) {
    phase_begin();
    if (!use_df_init(D, ca)) return;
    int t, rb;
    tile_rb(D.nrb, t, rb);
    const int lc = threadIdx.x % G, gc = t * G + lc;
    const bool valid = gc < ca->k;
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    for (int i = rb * D.rbs + threadIdx.x / G; i < i1; i += NTB / G) {
        float a = 0.0f, b = 0.0f, c = 0.0f, d = 0.0f;
        if (valid) {
            split_d2f(ca->xprev[(int64_t)i * ca->ld_prev + gc], a, b);
            if (ca->guess) split_d2f(ca->guess[(int64_t)i * ca->ld_guess + gc], c, d);
        }
        const size_t o = ((size_t)t * D.n + i) * G + lc;
        ph[o] = a;
        pl[o] = b;
        gh[o] = c;
        gl[o] = d;
    }
}

// sum_w (Ah + Al)[w, i] (xh + xl)[col[w, i]] over tile-major split parts, column lc
__device__ __forceinline__ double ell_df_split(const Depth& D, const float* Ah, const float* Al, const float* xh,
                                               const float* xl, int i, int lc, float* absum) {
    DfAcc acc;
    int j[WMAX];
    float ah[WMAX], al[WMAX];
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < D.W) {
            j[w] = __ldg(D.col + w * D.n + i);
            ah[w] = __ldg(Ah + w * D.n + i);
            al[w] = __ldg(Al + w * D.n + i);
        }
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < D.W) {
            const float h = xh[j[w] * G + lc], l = xl[j[w] * G + lc];
            acc.add(ah[w], al[w], h, l);
            if (absum) *absum += fabsf(ah[w]) * fabsf(h);
        }
    for (int w = WMAX; w < D.W; ++w) {
        const int jw = __ldg(D.col + w * D.n + i);
        const float aw = __ldg(Ah + w * D.n + i), h = xh[jw * G + lc];
        acc.add(aw, __ldg(Al + w * D.n + i), h, xl[jw * G + lc]);
        if (absum) *absum += fabsf(aw) * fabsf(h);
    }
    return acc.value();
}

// ---------------------------------------------------------------- set-up and final phases
// b = (1/dt) M x_prev + J0 sum_s b_s F_s, x0 = guess - g; FP64 form: r = b - L x0;
// FP32+refinement: b kept, the FP32 correction and Krylov vectors d, p, q zeroed.
// DF (FP64 form): M x_prev and L x0 as double-float products over the FP32 parts
// kb_split wrote (sp: x_prev high, low, guess high, low, each tile-major).
template <int MODE, bool DF = false>
__global__ void __launch_bounds__(NTB, DF ? 2 : 4) kb_init(Depth D, const CallArgs* __restrict__ ca, double inv_dt,
                                               const double* __restrict__ F, double J0, double* x64, double* r64,
                                               double* p64, double* q64, double* b64, float* z, double* part_bb,
                                               double* part_rr, double* part_ss, float* r32s, float* d32, float* p32,
                                               float* q32, const float* __restrict__ sp = nullptr) {
    static_assert(!DF || MODE == 0, "double-float products: FP64 form");
    phase_begin();
    if (MODE == 0 && sp && use_df_init(D, ca) != DF) return;  // the other variant runs this call
    int t, rb;
    tile_rb(D.nrb, t, rb);
    const int lc = threadIdx.x % G, gc = t * G + lc;
    const bool valid = gc < ca->k;
    double sg[3] = {0.0, 0.0, 0.0};
    if (valid) {
        const int64_t tt = ca->t0 + (int64_t)gc * ca->tstride;
        for (int q = 0; q < 3; ++q) sg[q] = ca->wave[3 * tt + q];
    }
    const double* xprev = ca->xprev;
    const double* guess = ca->guess;
    const double* g = ca->g;
    double bb[1] = {0.0}, rr[1] = {0.0}, ss[1] = {0.0};
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    for (int i = rb * D.rbs + threadIdx.x / G; i < i1; i += NTB / G) {
        double bi = 0.0, lx = 0.0, xi = 0.0;
        float alx = 0.0f;  // sum |L_ij| |x_j| of the rounding floor (an estimate: FP32)
        if (valid) {
            double mb = 0.0;
            if constexpr (DF) {  // g is null here (use_df_init)
                const size_t e = (size_t)D.n * G, tb = (size_t)t * e;
                mb = ell_df_split(D, D.M32, D.Mlo32, sp + tb, sp + e * gridDim.x / D.nrb + tb, i, lc, nullptr);
                if (guess)
                    lx = ell_df_split(D, D.L32, D.Llo32, sp + 2 * e * (gridDim.x / D.nrb) + tb,
                                      sp + 3 * e * (gridDim.x / D.nrb) + tb, i, lc, &alx);
            } else {
                for (int w = 0; w < D.W; ++w) {
                    const int64_t j = __ldg(D.col + w * D.n + i);
                    mb += __ldg(D.M64 + w * D.n + i) * xprev[j * ca->ld_prev + gc];
                    if (guess) {
                        double xj = guess[j * ca->ld_guess + gc];
                        if (g) xj -= g[j * ca->ld_g + gc];
                        lx += __ldg(D.L64 + w * D.n + i) * xj;
                        alx += fabsf(__ldg(D.L32 + w * D.n + i)) * abs_to_float(xj);
                    }
                }
            }
            bi = mb * inv_dt + J0 * (sg[0] * F[i] + sg[1] * F[D.n + i] + sg[2] * F[2 * D.n + i]);
            if (guess) {
                xi = guess[(int64_t)i * ca->ld_guess + gc];
                if (g) xi -= g[(int64_t)i * ca->ld_g + gc];
            }
        }
        const size_t o = ((size_t)t * D.n + i) * G + lc;
        x64[o] = xi;
        z[o] = 0.0f;
        if (MODE == 0) {
            const double ri = bi - lx;
            r64[o] = ri;
            r32s[o] = (float)ri;
            p64[o] = 0.0;
            q64[o] = 0.0;
            rr[0] += ri * ri;
            const float si = abs_to_float(bi) + alx;
            ss[0] += (double)(si * si);
        } else {
            b64[o] = bi;
            d32[o] = 0.0f;
            p32[o] = 0.0f;
            q32[o] = 0.0f;
        }
        bb[0] += bi * bi;
    }
    block_partial<1>(bb, part_bb);
    if (MODE == 0) {
        __syncthreads();
        block_partial<1>(rr, part_rr);
        __syncthreads();
        block_partial<1>(ss, part_ss);
    }
}

// x_out = x (+ d: the FP32 correction not yet folded into x) + g
__global__ void __launch_bounds__(NTB) kb_final(Depth D, const CallArgs* __restrict__ ca, const double* x64,
                                                const float* d32) {
    phase_begin();
    int t, rb;
    tile_rb(D.nrb, t, rb);
    const int lc = threadIdx.x % G, gc = t * G + lc;
    if (gc >= ca->k) return;
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    for (int i = rb * D.rbs + threadIdx.x / G; i < i1; i += NTB / G) {
        double xi = x64[((size_t)t * D.n + i) * G + lc];
        if (d32) xi += (double)d32[((size_t)t * D.n + i) * G + lc];
        if (ca->g) xi += ca->g[(int64_t)i * ca->ld_g + gc];
        ca->xout[(int64_t)i * ca->ld_out + gc] = xi;
    }
}

// ---------------------------------------------------------------- scalar (one-block) phases
constexpr int NSB = 1024;

// FP64 form: ||b||^2, ||r0||^2 -> active columns, loop condition.
// part_ss null: no rounding floor (Newton corrections start from delta = 0).
__global__ void __launch_bounds__(NSB) kb_scalar_init0(Cols st, const double* part_bb, const double* part_rr,
                                                      const double* part_ss, int nrb, int kpad,
                                                      const CallArgs* __restrict__ ca, cudaGraphConditionalHandle h,
                                                      int use_cond) {
    phase_begin();
    int any = 0;
    for (int c = threadIdx.x; c < kpad; c += NSB) {
        const double bb = col_total(part_bb, nrb, c), rr = col_total(part_rr, nrb, c);
        const double ss = part_ss ? col_total(part_ss, nrb, c) : 0.0;
        st.bb[c] = bb;
        st.ref[c] = bb;
        st.ss[c] = ss;
        st.gam[c] = 0.0;
        st.iters[c] = 0;
        st.bad[c] = (c < ca->k) && !(rr == rr && bb == bb && rr - rr == 0.0 && bb - bb == 0.0);
        // a guess that already solves the step to working precision is kept as it is
        const int a = (c < ca->k) && !(rr <= ca->tol2 * bb || rr <= ca->fl_acc2 * ss);
        st.act[c] = a;
        any |= a;
    }
    any = __syncthreads_or(any);
    for (int t = threadIdx.x; t < kpad / G; t += NSB) {
        int on = 0;
        for (int l = 0; l < G; ++l) on |= st.act[t * G + l];
        st.tact[t] = on;
    }
    if (threadIdx.x == 0) {
        st.ctr[0] = 0;
        st.ctr[2] = 0;
        st.ctr[3] = 0;
        if (use_cond) cudaGraphSetConditional(h, (any && ca->max_it > 0) ? 1u : 0u);
    }
}

// FP32+refinement: ||b||^2; every valid column starts with an FP64 residual update.
__global__ void __launch_bounds__(NSB) kb_scalar_init1(Cols st, const double* part_bb, int nrb, int kpad,
                                                      const CallArgs* __restrict__ ca) {
    phase_begin();
    for (int c = threadIdx.x; c < kpad; c += NSB) {
        const double bb = col_total(part_bb, nrb, c);
        st.bb[c] = bb;
        st.outer[c] = c < ca->k;
        st.upd[c] = c < ca->k;
        st.nup[c] = 0;
        st.stall[c] = 0;
        st.lastu[c] = 0;
        st.iters[c] = 0;
        st.act[c] = 0;
        st.gam[c] = 0.0;
        st.bad[c] = (c < ca->k) && !(bb - bb == 0.0);
    }
    if (threadIdx.x == 0) {
        st.ctr[0] = 0;
        st.ctr[2] = 0;
        st.ctr[3] = 0;
    }
}

// Per-column PCG scalars: one block per column tile (16 lanes per column add the
// tile's row-block partials in a fixed order).
__device__ __forceinline__ void tile_totals(const double* part, int nrb, int t, double* out) {
    static_assert(NTB == 16 * G, "tile_totals needs 16 lanes per column");
    const int c = threadIdx.x / 16, l = threadIdx.x % 16;
    double s = 0.0;
    for (int rb = l; rb < nrb; rb += 16) s += part[((size_t)t * nrb + rb) * G + c];
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (l == 0) out[c] = s;
    __syncthreads();
}

// (r, z) -> gamma, beta
__global__ void __launch_bounds__(NTB) kb_scalar_gamma(Cols st, const double* part, int nrb) {
    phase_begin();
    __shared__ double rz[G];
    tile_totals(part, nrb, blockIdx.x, rz);
    if (threadIdx.x < G) {
        const int c = blockIdx.x * G + threadIdx.x;
        const double gn = rz[threadIdx.x];
        st.beta[c] = (st.ctr[0] == 0 || st.gam[c] == 0.0) ? 0.0 : gn / st.gam[c];
        st.gam[c] = gn;
    }
}

// (p, q) -> alpha
__global__ void __launch_bounds__(NTB) kb_scalar_alpha(Cols st, const double* part, int nrb) {
    phase_begin();
    __shared__ double pq[G];
    tile_totals(part, nrb, blockIdx.x, pq);
    if (threadIdx.x < G) {
        const int c = blockIdx.x * G + threadIdx.x;
        const double v = pq[threadIdx.x];
        st.alpha[c] = (st.act[c] && v != 0.0) ? st.gam[c] / v : 0.0;
    }
}

// (r, r) -> convergence masks; the last tile block to finish (ticket in ctr[3],
// active tiles counted in ctr[2]) advances the iteration count and sets the loop
// condition.
__global__ void __launch_bounds__(NTB) kb_scalar_conv(Cols st, const double* part, int nrb,
                                                     const CallArgs* __restrict__ ca, int inner,
                                                     cudaGraphConditionalHandle h, int use_cond) {
    phase_begin();
    const double tol2 = inner ? ca->inner_tol2 : ca->tol2;
    __shared__ double rr[G];
    tile_totals(part, nrb, blockIdx.x, rr);
    int any = 0;
    if (threadIdx.x < G) {
        const int c = blockIdx.x * G + threadIdx.x;
        const double v = rr[threadIdx.x];
        if (st.act[c]) {
            st.iters[c] += 1;
            const bool floor = !inner && v <= ca->fl_stop2 * st.ss[c];
            if (!(v - v == 0.0)) st.bad[c] = 1;
            if (v <= tol2 * st.ref[c] || floor || !(v - v == 0.0)) st.act[c] = 0;
        }
        any = st.act[c];
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        st.tact[blockIdx.x] = any;
        if (any) atomicAdd(&st.ctr[2], 1);
        __threadfence();
        const unsigned ticket = atomicAdd(reinterpret_cast<unsigned*>(&st.ctr[3]), 1u);
        if (ticket == gridDim.x - 1) {
            __threadfence();
            const int active = atomicExch(&st.ctr[2], 0);
            st.ctr[3] = 0;
            const int it = st.ctr[0] + 1;
            st.ctr[0] = it;
            if (use_cond) cudaGraphSetConditional(h, (active && it < ca->max_it) ? 1u : 0u);
        }
    }
}

// FP32+refinement, after an FP32 iteration: a column whose FP32 residual has fallen
// by inner_tol since its last FP64 residual, or below the tolerance, gets an FP64
// update (the residual replacement of the reliable-update scheme); the last tile
// block advances the iteration count.
__global__ void __launch_bounds__(NTB) kb_scalar_conv_ru(Cols st, const double* part, int nrb,
                                                        const CallArgs* __restrict__ ca) {
    phase_begin();
    __shared__ double rr[G];
    tile_totals(part, nrb, blockIdx.x, rr);
    if (threadIdx.x < G) {
        const int c = blockIdx.x * G + threadIdx.x;
        const double v = rr[threadIdx.x];
        int u = 0;
        if (st.act[c]) {
            st.iters[c] += 1;
            if (!(v - v == 0.0)) {
                st.bad[c] = 1;
                st.act[c] = 0;
                st.outer[c] = 2;
            } else {
                u = v <= ca->inner_tol2 * st.ref[c] || v <= ca->tol2 * st.bb[c] ||
                    st.iters[c] - st.lastu[c] >= kMaxInner;
                if (u) st.prev[c] = v;  // the FP32 residual the FP64 one is compared with
            }
        }
        st.upd[c] = u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(reinterpret_cast<unsigned*>(&st.ctr[3]), 1u);
        if (ticket == gridDim.x - 1) {
            __threadfence();
            st.ctr[3] = 0;
            st.ctr[0] = st.ctr[0] + 1;
        }
    }
}

// FP32+refinement: decisions after the FP64 residual of the updated columns.  A
// column stops when ||r|| meets the tolerance or the rounding floor (the initial
// guess within the acceptance margin), fails when the residual is not finite, the
// updates exceed max_refine or three updates in a row took less than 10 % off ||r||
// above the acceptance margin; otherwise the FP32 iteration continues from the new
// residual.
// The last tile block sets the loop condition: columns left and iterations left.
__global__ void __launch_bounds__(NTB) kb_scalar_ru(Cols st, const double* part_rr, const double* part_ss, int nrb,
                                                   const CallArgs* __restrict__ ca, cudaGraphConditionalHandle h,
                                                   int use_cond) {
    phase_begin();
    __shared__ double rr[G], ss[G];
    tile_totals(part_rr, nrb, blockIdx.x, rr);
    tile_totals(part_ss, nrb, blockIdx.x, ss);
    int any = 0;
    if (threadIdx.x < G) {
        const int c = blockIdx.x * G + threadIdx.x;
        if (st.upd[c] && st.outer[c] == 1) {
            const double v = rr[threadIdx.x], sv = ss[threadIdx.x];
            const bool first = st.nup[c] == 0;
            const double fl2 = first ? ca->fl_acc2 : ca->fl_stop2;
            if (!(v - v == 0.0)) {
                st.bad[c] = 1;
                st.outer[c] = 2;
            } else if (v <= ca->tol2 * st.bb[c] || v <= fl2 * sv) {
                st.outer[c] = 0;
            } else {
                if (!first && v > 0.81 * st.ref[c]) st.stall[c] += 1;
                else st.stall[c] = 0;
                if (st.stall[c] >= 3) st.outer[c] = v <= ca->fl_acc2 * sv ? 0 : 2;
                else if (st.nup[c] > ca->max_refine) st.outer[c] = 2;
            }
            // the FP32 recurrence had drifted from the true residual by more than 2x:
            // its search direction no longer fits, restart it (beta = 0)
            if (!first && v > 4.0 * st.prev[c]) st.gam[c] = 0.0;
            st.nup[c] += 1;
            st.ref[c] = v;
            st.lastu[c] = st.iters[c];
            st.act[c] = st.outer[c] == 1;
        }
        any = st.act[c];
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        st.tact[blockIdx.x] = any;
        if (any) atomicAdd(&st.ctr[2], 1);
        __threadfence();
        const unsigned ticket = atomicAdd(reinterpret_cast<unsigned*>(&st.ctr[3]), 1u);
        if (ticket == gridDim.x - 1) {
            __threadfence();
            const int active = atomicExch(&st.ctr[2], 0);
            st.ctr[3] = 0;
            if (use_cond) cudaGraphSetConditional(h, (active && st.ctr[0] < ca->max_it) ? 1u : 0u);
        }
    }
}

// statuses and iteration totals into the context counters
__global__ void __launch_bounds__(NSB) kb_scalar_final(Cols st, int kpad, const CallArgs* __restrict__ ca, int mode,
                                                      unsigned long long* iter_sum, int* worst) {
    phase_begin();
    for (int c = threadIdx.x; c < kpad && c < ca->k; c += NSB) {
        const int failed = mode == 0 ? st.act[c] : st.outer[c] != 0;
        if (st.bad[c]) atomicMin(worst, (int)MG_ENONFINITE);
        else if (failed) atomicMin(worst, (int)MG_ECG_MAXIT);
        atomicAdd(iter_sum, (unsigned long long)st.iters[c]);
    }
}

template <class A, class X>
__device__ __forceinline__ A widen(X x) { return (A)x; }
template <>
__device__ __forceinline__ double widen<double, float>(float x) { return f2d_int(x); }

// ELL values: one value per entry shared by all columns (PC = false), or per
// column (PC = true): entry (w, i) of tile t, column c at ((t W n + w n + i) G + c).
template <bool PC, class VAL>
__device__ __forceinline__ const VAL* tile_vals(const VAL* p, const Depth& D, int t) {
    return PC ? p + (size_t)t * D.W * D.n * G : p;
}

// ELL row product acc[e] = sum_w val[w, i] v[col[w, i]][c0 + e], the operand
// widened by widen<A>(); val from tile_vals<PC>()
template <int V, class A, class VAL, class X, bool PC = false>
__device__ __forceinline__ void ell_vec_w(const int32_t* __restrict__ col, const VAL* __restrict__ val, int n, int W,
                                          int i, const X* v, int c0, A (&acc)[V]) {
    constexpr int NV = PC ? V : 1;
#pragma unroll
    for (int e = 0; e < V; ++e) acc[e] = 0;
    int32_t j[WMAX];
    VAL a[WMAX][NV];
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < W) {
            j[w] = __ldg(col + w * n + i);
            if constexpr (PC) vld<VAL, V>(val + ((size_t)w * n + i) * G + c0, a[w]);
            else a[w][0] = __ldg(val + w * n + i);
        }
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < W) {
            X xv[V];
            vld<X, V>(v + j[w] * G + c0, xv);
#pragma unroll
            for (int e = 0; e < V; ++e) acc[e] += (A)a[w][PC ? e : 0] * widen<A, X>(xv[e]);
        }
    for (int w = WMAX; w < W; ++w) {
        X xv[V];
        vld<X, V>(v + __ldg(col + w * n + i) * G + c0, xv);
        VAL aw[NV];
        if constexpr (PC) vld<VAL, V>(val + ((size_t)w * n + i) * G + c0, aw);
        else aw[0] = __ldg(val + w * n + i);
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] += (A)aw[PC ? e : 0] * widen<A, X>(xv[e]);
    }
}

// Jacobi scaling 1/diag of row i for columns c0 .. c0+V-1
template <bool PC, int V>
__device__ __forceinline__ void dinv_of(const Depth& D, int t, int i, int c0, float (&d)[V]) {
    if constexpr (PC) {
        vld<float, V>(D.dinv32 + ((size_t)t * D.n + i) * G + c0, d);
    } else {
        const float x = __ldg(D.dinv32 + i);
#pragma unroll
        for (int e = 0; e < V; ++e) d[e] = x;
    }
}

// ---------------------------------------------------------------- multigrid phases (FP32, float4 lanes)
constexpr int VF = 4;
constexpr int TPRF = G / VF;       // threads per row
constexpr int RPPF = NTB / TPRF;   // rows per pass

#define ROWS_F(D, t, rb, i)                                   \
    int t, rb;                                                \
    tile_rb((D).nrb, t, rb);                                  \
    if (!tile_on((D).tact, t)) return;                        \
    const int c0 = (threadIdx.x % TPRF) * VF;                 \
    const int _i1 = min((D).n, (rb + 1) * (D).rbs);           \
    for (int i = rb * (D).rbs + threadIdx.x / TPRF; i < _i1; i += RPPF)

// sweep weight: w, divided by the device-side spectral bound *lam when given
__device__ __forceinline__ float sweep_weight(float w, const unsigned* lam) {
    return lam ? w / __uint_as_float(__ldg(lam)) : w;
}

// Launch shape of the gather-bound smoothing and residual-update kernels.  A thread
// may take MG_SRB rows per batch, the loads of all of them (indices, values,
// gathered neighbours) issued before any result is stored, so that their
// latencies overlap; and MG_MINB_S (shared operators) or MG_MINB_PC (per-column
// Newton Jacobians, four values per entry and lane) blocks of 256 threads must fit
// an SM, which caps the registers of a thread.  Measured on GB300 (one batched FP64
// step to 1e-13, 18,240 DOFs x 256 columns / 73,344 x 1,024): one row and 4 blocks
// (64 registers) 5.40 / 76.3 ms; one row and 5 blocks (48 registers, spilling)
// 6.60 / 92.6 ms; two rows and 3 blocks 6.36 / 84.5 ms; two rows and 4 blocks
// 6.77 / 91.8 ms; four rows and 2 blocks 6.56 / 104.7 ms.  Spills, not the
// latency of one row, were the cost.
#ifndef MG_SRB
#define MG_SRB 1
#endif
#ifndef MG_MINB_S
#define MG_MINB_S 4
#endif
#ifndef MG_MINB_PC
#define MG_MINB_PC 3
#endif
template <bool PC>
__host__ __device__ constexpr int srb() { return PC ? 1 : MG_SRB; }
template <bool PC>
__host__ __device__ constexpr int minb_s() { return PC ? MG_MINB_PC : MG_MINB_S; }

// x = w D^-1 r, s = r - w (L D^-1) r
template <class RT, bool PC>
__global__ void __launch_bounds__(NTB, minb_s<PC>()) kb_smooth_first(Depth D, const RT* rin_base, float w0,
                                                                     const unsigned* lam) {
    constexpr int SRB = srb<PC>();
    phase_begin();
    const float w = sweep_weight(w0, lam);
    int t, rb;
    tile_rb(D.nrb, t, rb);
    if (!tile_on(D.tact, t)) return;
    const int c0 = (threadIdx.x % TPRF) * VF;
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    const RT* rin = tv(rin_base, D.n, t);
    float* x = tv(D.x, D.n, t);
    float* sa = tv(D.sa, D.n, t);
    for (int i0 = rb * D.rbs + threadIdx.x / TPRF; i0 < i1; i0 += RPPF * SRB) {
        RT rv[SRB][VF];
        float acc[SRB][VF], di[SRB][VF];
#pragma unroll
        for (int q = 0; q < SRB; ++q) {
            const int i = i0 + q * RPPF;
            if (i < i1) {
                vld<RT, VF>(rin + i * G + c0, rv[q]);
                ell_vec_w<VF, float, float, RT, PC>(D.col, tile_vals<PC>(D.LD32, D, t), D.n, D.W, i, rin, c0,
                                                    acc[q]);
                dinv_of<PC>(D, t, i, c0, di[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < SRB; ++q) {
            const int i = i0 + q * RPPF;
            if (i < i1) {
                float xo[VF], so[VF];
#pragma unroll
                for (int e = 0; e < VF; ++e) {
                    xo[e] = w * di[q][e] * (float)rv[q][e];
                    so[e] = (float)rv[q][e] - w * acc[q][e];
                }
                vst<float, VF>(x + i * G + c0, xo);
                vst<float, VF>(sa + i * G + c0, so);
            }
        }
    }
}

// x += w D^-1 s; s' = s - w (L D^-1) s if dst is given (not on a level's last sweep);
// partial (r, x) if rtop is given (last sweep on the finest level)
template <class RT, bool PC>
__global__ void __launch_bounds__(NTB, minb_s<PC>()) kb_smooth(Depth D, const float* src_base, float* dst_base,
                                                               const RT* rtop_base, float w0, const unsigned* lam,
                                                               double* part) {
    constexpr int SRB = srb<PC>();
    phase_begin();
    const float w = sweep_weight(w0, lam);
    // (r, x) of a thread's few rows: FP32 sums for shared operators (linear steps,
    // where |r_i x_i| ~ r_i^2 / L_ii stays far inside the FP32 range); FP64 for
    // Newton corrections, whose residuals near convergence are so small that FP32
    // products of r and x would underflow
    using RZ = typename std::conditional<PC, double, float>::type;
    RZ rz[VF] = {};
    int t, rb;
    tile_rb(D.nrb, t, rb);
    if (!tile_on(D.tact, t)) return;
    const int c0 = (threadIdx.x % TPRF) * VF;
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    const float* src = tv(src_base, D.n, t);
    float* x = tv(D.x, D.n, t);
    float* dst = dst_base ? tv(dst_base, D.n, t) : nullptr;
    const RT* rtop = rtop_base ? tv(rtop_base, D.n, t) : nullptr;
    for (int i0 = rb * D.rbs + threadIdx.x / TPRF; i0 < i1; i0 += RPPF * SRB) {
        float sv[SRB][VF], xv[SRB][VF], di[SRB][VF], acc[SRB][VF];
        RT rv[SRB][VF];
#pragma unroll
        for (int q = 0; q < SRB; ++q) {
            const int i = i0 + q * RPPF;
            if (i < i1) {
                vld<float, VF>(src + i * G + c0, sv[q]);
                vld<float, VF>(x + i * G + c0, xv[q]);
                dinv_of<PC>(D, t, i, c0, di[q]);
                if (rtop) vld<RT, VF>(rtop + i * G + c0, rv[q]);
                // the next residual is needed unless this is the last sweep
                if (dst)
                    ell_vec_w<VF, float, float, float, PC>(D.col, tile_vals<PC>(D.LD32, D, t), D.n, D.W, i, src, c0,
                                                           acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < SRB; ++q) {
            const int i = i0 + q * RPPF;
            if (i < i1) {
                float xo[VF];
#pragma unroll
                for (int e = 0; e < VF; ++e) xo[e] = xv[q][e] + w * di[q][e] * sv[q][e];
                vst<float, VF>(x + i * G + c0, xo);
                if (rtop) {
#pragma unroll
                    for (int e = 0; e < VF; ++e) rz[e] += widen<RZ, RT>(rv[q][e]) * widen<RZ, float>(xo[e]);
                }
                if (dst) {
                    float so[VF];
#pragma unroll
                    for (int e = 0; e < VF; ++e) so[e] = sv[q][e] - w * acc[q][e];
                    vst<float, VF>(dst + i * G + c0, so);
                }
            }
        }
    }
    if (rtop_base) {
        double rzd[VF];
#pragma unroll
        for (int e = 0; e < VF; ++e) rzd[e] = widen<double, RZ>(rz[e]);
        block_partial<VF>(rzd, part);
    }
}

// Two consecutive smoothing sweeps in one launch, for operators shared by all
// columns.  Sweep a: x1 = x0 + wa D^-1 s0, s1 = s0 - wa (L D^-1) s0; sweep b:
// x2 = x1 + wb D^-1 s1 and, unless dst is null, s2 = s1 - wb (L D^-1) s1.  FIRST:
// the depth's first sweep, x0 = 0 and s0 the V-cycle's input residual.  A block
// owns rows [a, a + R) of CW columns of one tile.  It forms s1 in shared memory on
// every row within the operator's bandwidth H of its own rows, [a - H, a + R + H),
// reading s0 through L2, so that the second sweep gathers s1 from shared memory and
// s1 never leaves the SM; the halo rows' first sweep is done by both neighbouring
// blocks.  STAGE: s0 itself is first copied into shared memory on the rows within
// 2H of the block's rows (coalesced streaming loads), so that the first sweep too
// gathers from shared memory.  Same arithmetic, in the same order, as
// kb_smooth_first / kb_smooth.
constexpr int NT2 = 512;

// row product acc[e] = sum_w LD[w, i] v[col[w, i] - lo][e] over a shared-memory vector
template <int TPR>
__device__ __forceinline__ void ell_row_sh(const Depth& D, int i, const float4* v, int lo, int l, float (&acc)[VF]) {
#pragma unroll
    for (int e = 0; e < VF; ++e) acc[e] = 0.0f;
    int j[WMAX];
    float a[WMAX];
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < D.W) {
            j[w] = __ldg(D.col + w * D.n + i);
            a[w] = __ldg(D.LD32 + w * D.n + i);
        }
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < D.W) {
            const float4 sj = v[(j[w] - lo) * TPR + l];
            acc[0] += a[w] * sj.x;
            acc[1] += a[w] * sj.y;
            acc[2] += a[w] * sj.z;
            acc[3] += a[w] * sj.w;
        }
    for (int w = WMAX; w < D.W; ++w) {
        const float4 sj = v[(__ldg(D.col + w * D.n + i) - lo) * TPR + l];
        const float aw = __ldg(D.LD32 + w * D.n + i);
        acc[0] += aw * sj.x;
        acc[1] += aw * sj.y;
        acc[2] += aw * sj.z;
        acc[3] += aw * sj.w;
    }
}

template <int CW, bool FIRST, bool STAGE>
__global__ void __launch_bounds__(NT2, 2) kb_smooth2(Depth D, const float* s0_base, float* dst_base, float wa,
                                                     float wb) {
    // shared memory: STAGE: s0 on (R + 4H) rows, then s1 on (R + 2H) rows; else s1 only
    extern __shared__ float4 sh2[];
    constexpr int TPR = CW / VF, RPP = NT2 / TPR, NSUB = G / CW;
    phase_begin();
    const int rb = blockIdx.x % D.f_nrb;
    const int grp = blockIdx.x / D.f_nrb;
    const int t = grp / NSUB;
    if (!tile_on(D.tact, t)) return;
    const int l = threadIdx.x % TPR;
    const int c0 = (grp % NSUB) * CW + l * VF;
    const int a = rb * D.f_R, b = min(D.n, a + D.f_R);
    const int lo = max(0, a - D.f_H), hi = min(D.n, b + D.f_H);
    const int lo0 = max(0, a - 2 * D.f_H), hi0 = min(D.n, b + 2 * D.f_H);
    const float* s0 = tv(s0_base, D.n, t);
    float4* s0sh = sh2;
    float4* s1sh = STAGE ? sh2 + (size_t)(D.f_R + 4 * D.f_H) * TPR : sh2;
    if constexpr (STAGE) {
        for (int i = lo0 + (int)threadIdx.x / TPR; i < hi0; i += RPP) {
            float sv[VF];
            vld<float, VF>(s0 + i * G + c0, sv);
            s0sh[(i - lo0) * TPR + l] = make_float4(sv[0], sv[1], sv[2], sv[3]);
        }
        __syncthreads();
    }
    for (int i = lo + (int)threadIdx.x / TPR; i < hi; i += RPP) {
        float sv[VF], acc[VF];
        if constexpr (STAGE) {
            const float4 v = s0sh[(i - lo0) * TPR + l];
            sv[0] = v.x;
            sv[1] = v.y;
            sv[2] = v.z;
            sv[3] = v.w;
            ell_row_sh<TPR>(D, i, s0sh, lo0, l, acc);
        } else {
            vld<float, VF>(s0 + i * G + c0, sv);
            ell_vec_w<VF, float, float, float, false>(D.col, D.LD32, D.n, D.W, i, s0, c0, acc);
        }
        float4 o;
        o.x = sv[0] - wa * acc[0];
        o.y = sv[1] - wa * acc[1];
        o.z = sv[2] - wa * acc[2];
        o.w = sv[3] - wa * acc[3];
        s1sh[(i - lo) * TPR + l] = o;
    }
    __syncthreads();
    float* x = tv(D.x, D.n, t);
    float* dst = dst_base ? tv(dst_base, D.n, t) : nullptr;
    for (int i = a + (int)threadIdx.x / TPR; i < b; i += RPP) {
        const float4 s1v = s1sh[(i - lo) * TPR + l];
        const float s1[VF] = {s1v.x, s1v.y, s1v.z, s1v.w};
        float sv[VF], xv[VF];
        if constexpr (STAGE) {
            const float4 v = s0sh[(i - lo0) * TPR + l];
            sv[0] = v.x;
            sv[1] = v.y;
            sv[2] = v.z;
            sv[3] = v.w;
        } else {
            vld<float, VF>(s0 + i * G + c0, sv);
        }
        const float di = __ldg(D.dinv32 + i);
        if constexpr (FIRST) {
#pragma unroll
            for (int e = 0; e < VF; ++e) xv[e] = wa * di * sv[e];
        } else {
            vld<float, VF>(x + i * G + c0, xv);
#pragma unroll
            for (int e = 0; e < VF; ++e) xv[e] = xv[e] + wa * di * sv[e];
        }
#pragma unroll
        for (int e = 0; e < VF; ++e) xv[e] = xv[e] + wb * di * s1[e];
        vst<float, VF>(x + i * G + c0, xv);
        if (dst) {
            float acc[VF];
            ell_row_sh<TPR>(D, i, s1sh, lo, l, acc);
            float so[VF];
#pragma unroll
            for (int e = 0; e < VF; ++e) so[e] = s1[e] - wb * acc[e];
            vst<float, VF>(dst + i * G + c0, so);
        }
    }
}

// r_c = P^T s over the coarse rows (grid over the coarse depth's row blocks)
__global__ void __launch_bounds__(NTB, MG_MINB_F) kb_restrict(Depth D, Depth C, const float* src_base) {
    phase_begin();
    ROWS_F(C, t, rb, ic) {
        const float* src = tv(src_base, D.n, t);
        float acc[VF] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int w = 0; w < D.rt_W; ++w) {
            const int j = __ldg(D.rt_col + w * C.n + ic);
            const float a = __ldg(D.rt_w + w * C.n + ic);
            float xv[VF];
            vld<float, VF>(src + j * G + c0, xv);
#pragma unroll
            for (int e = 0; e < VF; ++e) acc[e] += a * xv[e];
        }
        vst<float, VF>(tv(C.r, C.n, t) + ic * G + c0, acc);
    }
}

// y = P x_c, x += y  (x_c = sum of `parts` partial vectors pstride apart)
__global__ void __launch_bounds__(NTB, MG_MINB_F) kb_prolong(Depth D, Depth C, int parts, size_t pstride) {
    phase_begin();
    ROWS_F(D, t, rb, i) {
        const float* xc = tv(C.x, C.n, t);
        float yv[VF] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int p = __ldg(D.par + q * D.n + i);
            if (p >= 0) {
                const float wq = __ldg(D.pw + q * D.n + i);
                float xv[VF];
                vld<float, VF>(xc + p * G + c0, xv);
                for (int sp = 1; sp < parts; ++sp) {
                    float xs[VF];
                    vld<float, VF>(xc + sp * pstride + p * G + c0, xs);
#pragma unroll
                    for (int e = 0; e < VF; ++e) xv[e] += xs[e];
                }
#pragma unroll
                for (int e = 0; e < VF; ++e) yv[e] += wq * xv[e];
            }
        }
        float* x = tv(D.x, D.n, t);
        float xv[VF];
        vld<float, VF>(x + i * G + c0, xv);
#pragma unroll
        for (int e = 0; e < VF; ++e) xv[e] += yv[e];
        vst<float, VF>(x + i * G + c0, xv);
        vst<float, VF>(tv(D.y, D.n, t) + i * G + c0, yv);
    }
}

// Prolongation and residual update in one launch, for operators shared by all
// columns: y = P x_c, x += y, s -= L y.  A block owns rows [a, a + R) of CW
// columns of one tile (the kb_smooth2 shape) and forms y in shared memory on the
// rows within the bandwidth H of them, so y never leaves the SM.  Same arithmetic,
// in the same order, as kb_prolong followed by kb_resupdate.
template <int CW>
__global__ void __launch_bounds__(NT2, 2) kb_prolong_res(Depth D, Depth C, int parts, size_t pstride,
                                                         float* s_base) {
    extern __shared__ float4 ysh[];  // (R + 2H) rows x CW floats
    constexpr int TPR = CW / VF, RPP = NT2 / TPR, NSUB = G / CW;
    phase_begin();
    const int rb = blockIdx.x % D.f_nrb;
    const int grp = blockIdx.x / D.f_nrb;
    const int t = grp / NSUB;
    if (!tile_on(D.tact, t)) return;
    const int l = threadIdx.x % TPR;
    const int c0 = (grp % NSUB) * CW + l * VF;
    const int a = rb * D.f_R, b = min(D.n, a + D.f_R);
    const int lo = max(0, a - D.f_H), hi = min(D.n, b + D.f_H);
    const float* xc = tv(C.x, C.n, t);
    for (int i = lo + (int)threadIdx.x / TPR; i < hi; i += RPP) {
        float yv[VF] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int p = __ldg(D.par + q * D.n + i);
            if (p >= 0) {
                const float wq = __ldg(D.pw + q * D.n + i);
                float xv[VF];
                vld<float, VF>(xc + p * G + c0, xv);
                for (int sp = 1; sp < parts; ++sp) {
                    float xs[VF];
                    vld<float, VF>(xc + sp * pstride + p * G + c0, xs);
#pragma unroll
                    for (int e = 0; e < VF; ++e) xv[e] += xs[e];
                }
#pragma unroll
                for (int e = 0; e < VF; ++e) yv[e] += wq * xv[e];
            }
        }
        ysh[(i - lo) * TPR + l] = make_float4(yv[0], yv[1], yv[2], yv[3]);
    }
    __syncthreads();
    float* x = tv(D.x, D.n, t);
    float* s = tv(s_base, D.n, t);
    for (int i = a + (int)threadIdx.x / TPR; i < b; i += RPP) {
        const float4 yi = ysh[(i - lo) * TPR + l];
        const float yv[VF] = {yi.x, yi.y, yi.z, yi.w};
        float xv[VF], sv[VF];
        vld<float, VF>(x + i * G + c0, xv);
        vld<float, VF>(s + i * G + c0, sv);
#pragma unroll
        for (int e = 0; e < VF; ++e) xv[e] += yv[e];
        vst<float, VF>(x + i * G + c0, xv);
        float acc[VF] = {0.0f, 0.0f, 0.0f, 0.0f};
        int j[WMAX];
        float v[WMAX];
#pragma unroll
        for (int w = 0; w < WMAX; ++w)
            if (w < D.W) {
                j[w] = __ldg(D.col + w * D.n + i);
                v[w] = __ldg(D.L32 + w * D.n + i);
            }
#pragma unroll
        for (int w = 0; w < WMAX; ++w)
            if (w < D.W) {
                const float4 yj = ysh[(j[w] - lo) * TPR + l];
                acc[0] += v[w] * yj.x;
                acc[1] += v[w] * yj.y;
                acc[2] += v[w] * yj.z;
                acc[3] += v[w] * yj.w;
            }
        for (int w = WMAX; w < D.W; ++w) {
            const float4 yj = ysh[(__ldg(D.col + w * D.n + i) - lo) * TPR + l];
            const float vw = __ldg(D.L32 + w * D.n + i);
            acc[0] += vw * yj.x;
            acc[1] += vw * yj.y;
            acc[2] += vw * yj.z;
            acc[3] += vw * yj.w;
        }
#pragma unroll
        for (int e = 0; e < VF; ++e) sv[e] -= acc[e];
        vst<float, VF>(s + i * G + c0, sv);
    }
}

// s -= L y
template <bool PC>
__global__ void __launch_bounds__(NTB, minb_s<PC>()) kb_resupdate(Depth D, float* s_base) {
    constexpr int SRB = srb<PC>();
    phase_begin();
    int t, rb;
    tile_rb(D.nrb, t, rb);
    if (!tile_on(D.tact, t)) return;
    const int c0 = (threadIdx.x % TPRF) * VF;
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    float* s = tv(s_base, D.n, t);
    const float* y = tv(D.y, D.n, t);
    for (int i0 = rb * D.rbs + threadIdx.x / TPRF; i0 < i1; i0 += RPPF * SRB) {
        float acc[SRB][VF], sv[SRB][VF];
#pragma unroll
        for (int q = 0; q < SRB; ++q) {
            const int i = i0 + q * RPPF;
            if (i < i1) {
                ell_vec_w<VF, float, float, float, PC>(D.col, tile_vals<PC>(D.L32, D, t), D.n, D.W, i, y, c0, acc[q]);
                vld<float, VF>(s + i * G + c0, sv[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < SRB; ++q) {
            const int i = i0 + q * RPPF;
            if (i < i1) {
#pragma unroll
                for (int e = 0; e < VF; ++e) sv[q][e] -= acc[q][e];
                vst<float, VF>(s + i * G + c0, sv[q]);
            }
        }
    }
}

// coarsest level: x = A^-1 r, a dense contraction on the tensor cores.  Warp-level
// m16n8k8 TF32 MMAs with FP32 accumulation; each operand is split into a TF32 high
// part and a TF32 remainder and three products (hi*hi + hi*lo + lo*hi) are
// accumulated, which keeps FP32-level accuracy.  Block: 4 warps = 64 rows x one
// 16-column tile; a warp owns 16 rows x 16 columns (two n8 fragments).
__device__ __forceinline__ unsigned tf32_of(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
    hi = tf32_of(x);
    lo = tf32_of(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int BASE_KSPLIT = 4;  // K splits of the dense base solve (partials summed by the prolongation)

// A block computes 64 rows x TB column tiles (TB x 16 columns) over one K range,
// staging BKT columns of A's 64-row slice and BKT rows of r per step, so one A
// slice serves TB tiles.  The K range is split over `ks` blocks per output block
// (grid = ks x row blocks x column groups, split fastest); split s writes its
// partial product to x_base + s * pstride and the consumer adds the ks partials
// in order.
template <class RT, int TB, int BKT>
__global__ void __launch_bounds__(128) kb_base_dense(int n0, const float* __restrict__ A, const RT* r_base,
                                                     float* x_base, int ntile, int ks, size_t pstride) {
    phase_begin();
    __shared__ __align__(16) float As[64][BKT + 4];    // +4: conflict-free fragment reads
    __shared__ __align__(16) float Bs[BKT][TB * G + 8];  // +8: conflict-free fragment reads
    const int nrb = (n0 + 63) / 64;
    const int split = blockIdx.x % ks, bt = blockIdx.x / ks;
    const int cg = bt / nrb, ib = bt % nrb;
    const int kspan = ((n0 + ks - 1) / ks + BKT - 1) / BKT * BKT;
    const int kbeg = split * kspan, kend = min(n0, kbeg + kspan);
    x_base += (size_t)split * pstride;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tig = lane & 3;
    float acc[2 * TB][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += BKT) {
        // stage A[ib*64 .. +64][k0 .. k0+BKT) and r[k0 .. k0+BKT][tiles cg*TB .. +TB)
        for (int q = threadIdx.x; q < 64 * BKT; q += 128) {
            const int rr = q / BKT, kk = q % BKT;
            const int gi = ib * 64 + rr, gk = k0 + kk;
            As[rr][kk] = (gi < n0 && gk < kend) ? __ldg(A + (size_t)gi * n0 + gk) : 0.0f;
        }
        for (int q = threadIdx.x; q < BKT * TB * G; q += 128) {
            const int kk = q / (TB * G), cc = q % (TB * G);
            const int t = cg * TB + cc / G, gk = k0 + kk;
            Bs[kk][cc] = (gk < kend && t < ntile) ? (float)r_base[((size_t)t * n0 + gk) * G + cc % G] : 0.0f;
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < BKT; kk += 8) {
            const int ra = warp * 16 + g;
            unsigned ahi[4], alo[4];
            split_tf32(As[ra][kk + tig], ahi[0], alo[0]);
            split_tf32(As[ra + 8][kk + tig], ahi[1], alo[1]);
            split_tf32(As[ra][kk + tig + 4], ahi[2], alo[2]);
            split_tf32(As[ra + 8][kk + tig + 4], ahi[3], alo[3]);
#pragma unroll
            for (int f = 0; f < 2 * TB; ++f) {
                unsigned bh0, bl0, bh1, bl1;
                split_tf32(Bs[kk + tig][f * 8 + g], bh0, bl0);
                split_tf32(Bs[kk + tig + 4][f * 8 + g], bh1, bl1);
                mma_tf32(acc[f], ahi, bh0, bh1);
                mma_tf32(acc[f], ahi, bl0, bl1);
                mma_tf32(acc[f], alo, bh0, bh1);
            }
        }
        __syncthreads();
    }
    const int ra = ib * 64 + warp * 16 + g, rb8 = ra + 8;
#pragma unroll
    for (int f = 0; f < 2 * TB; ++f) {
        const int t = cg * TB + f / 2;
        if (t >= ntile) continue;
        float* xb = x_base + (size_t)t * n0 * G;
        const int cc = (f % 2) * 8 + tig * 2;
        if (ra < n0) {
            xb[(size_t)ra * G + cc] = acc[f][0];
            xb[(size_t)ra * G + cc + 1] = acc[f][1];
        }
        if (rb8 < n0) {
            xb[(size_t)rb8 * G + cc] = acc[f][2];
            xb[(size_t)rb8 * G + cc + 1] = acc[f][3];
        }
    }
}

// The same contraction on the CUDA cores in FP32 (same block shape, K split and
// partial outputs as kb_base_dense).  A thread owns 4 rows x CT columns of the
// block's 64 x TB*16 outputs; the A slice is staged transposed so that a thread
// reads its 4 rows of one k as one float4, the r slice row-major so that it reads
// its CT columns as float4s.  When the base size is a multiple of 4 the slices
// are fetched as float4s into registers one step ahead, so that their global
// latency overlaps the previous step's arithmetic; otherwise element by element.
template <class RT, int TB, int BKT>
__global__ void __launch_bounds__(128) kb_base_cc(int n0, const float* __restrict__ A, const RT* r_base, float* x_base,
                                                  int ntile, int ks, size_t pstride) {
    constexpr int NC = TB * G;                 // columns per block
    constexpr int CT = NC / 8;                 // columns per thread (8 column groups)
    constexpr int AQ = 64 * BKT / 4 / 128;     // float4s of the A slice per thread
    constexpr int BQ = BKT * NC / 4 / 128;     // float4s of the r slice per thread
    static_assert(AQ >= 1 && BQ >= 1 && BKT % 4 == 0, "slice shape");
    phase_begin();
    __shared__ __align__(16) float At[BKT][64 + 4];
    __shared__ __align__(16) float Bs[BKT][NC];
    const int nrb = (n0 + 63) / 64;
    const int split = blockIdx.x % ks, bt = blockIdx.x / ks;
    const int cg = bt / nrb, ib = bt % nrb;
    const int kspan = ((n0 + ks - 1) / ks + BKT - 1) / BKT * BKT;
    const int kbeg = split * kspan, kend = min(n0, kbeg + kspan);
    x_base += (size_t)split * pstride;
    const int r0 = (threadIdx.x / 8) * 4, c0 = (threadIdx.x % 8) * CT;
    float acc[4][CT] = {};
    auto compute = [&]() {
#pragma unroll 4
        for (int kk = 0; kk < BKT; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&At[kk][r0]);
            float b[CT];
            if constexpr (CT % 4 == 0) {
#pragma unroll
                for (int q = 0; q < CT; q += 4) {
                    const float4 v = *reinterpret_cast<const float4*>(&Bs[kk][c0 + q]);
                    b[q] = v.x;
                    b[q + 1] = v.y;
                    b[q + 2] = v.z;
                    b[q + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < CT; q += 2) {
                    const float2 v = *reinterpret_cast<const float2*>(&Bs[kk][c0 + q]);
                    b[q] = v.x;
                    b[q + 1] = v.y;
                }
            }
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                acc[0][c] += a.x * b[c];
                acc[1][c] += a.y * b[c];
                acc[2][c] += a.z * b[c];
                acc[3][c] += a.w * b[c];
            }
        }
    };
    if (std::is_same<RT, float>::value && (n0 & 3) == 0) {
        // k ranges start at multiples of BKT and end at n0 or such a multiple: a
        // float4 of A or r lies wholly inside or wholly outside [kbeg, kend)
        float4 ra[AQ], rv[BQ];
        auto load = [&](int k0) {
#pragma unroll
            for (int u = 0; u < AQ; ++u) {
                const int q = threadIdx.x + u * 128;
                const int rr = q / (BKT / 4), gk = k0 + 4 * (q % (BKT / 4)), gi = ib * 64 + rr;
                ra[u] = (gi < n0 && gk < kend) ? __ldg(reinterpret_cast<const float4*>(A + (size_t)gi * n0 + gk))
                                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < BQ; ++u) {
                const int q = threadIdx.x + u * 128;
                const int gk = k0 + q / (NC / 4), cc = 4 * (q % (NC / 4)), t = cg * TB + cc / G;
                rv[u] = (gk < kend && t < ntile)
                            ? *reinterpret_cast<const float4*>(r_base + ((size_t)t * n0 + gk) * G + cc % G)
                            : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        };
        load(kbeg);
        for (int k0 = kbeg; k0 < kend; k0 += BKT) {
#pragma unroll
            for (int u = 0; u < AQ; ++u) {
                const int q = threadIdx.x + u * 128;
                const int rr = q / (BKT / 4), k4 = 4 * (q % (BKT / 4));
                At[k4][rr] = ra[u].x;
                At[k4 + 1][rr] = ra[u].y;
                At[k4 + 2][rr] = ra[u].z;
                At[k4 + 3][rr] = ra[u].w;
            }
#pragma unroll
            for (int u = 0; u < BQ; ++u) {
                const int q = threadIdx.x + u * 128;
                *reinterpret_cast<float4*>(&Bs[q / (NC / 4)][4 * (q % (NC / 4))]) = rv[u];
            }
            __syncthreads();
            if (k0 + BKT < kend) load(k0 + BKT);
            compute();
            __syncthreads();
        }
    } else {
        for (int k0 = kbeg; k0 < kend; k0 += BKT) {
            for (int q = threadIdx.x; q < 64 * BKT; q += 128) {
                const int rr = q / BKT, kk = q % BKT;
                const int gi = ib * 64 + rr, gk = k0 + kk;
                At[kk][rr] = (gi < n0 && gk < kend) ? __ldg(A + (size_t)gi * n0 + gk) : 0.0f;
            }
            for (int q = threadIdx.x; q < BKT * NC; q += 128) {
                const int kk = q / NC, cc = q % NC;
                const int t = cg * TB + cc / G, gk = k0 + kk;
                Bs[kk][cc] = (gk < kend && t < ntile) ? (float)r_base[((size_t)t * n0 + gk) * G + cc % G] : 0.0f;
            }
            __syncthreads();
            compute();
            __syncthreads();
        }
    }
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
        const int gi = ib * 64 + r0 + rr;
        if (gi >= n0) continue;
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            const int cc = c0 + c, t = cg * TB + cc / G;
            if (t < ntile) x_base[((size_t)t * n0 + gi) * G + cc % G] = acc[rr][c];
        }
    }
}

// launch with the programmatic-dependent-launch attribute (see phase_begin)
template <typename... KArgs, typename... Args>
void pdl_launch(void (*kern)(KArgs...), unsigned g, unsigned b, size_t smem, cudaStream_t s, Args... args) {
#if MG_PDL
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g);
    cfg.blockDim = dim3(b);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    MG_CUDA(cudaLaunchKernelEx(&cfg, kern, (KArgs)args...));
#else
    kern<<<g, b, smem, s>>>((KArgs)args...);
#endif
}

// launch the dense base solve with TB tiles per block for ntile tiles
#ifndef MG_BASE_TB
#define MG_BASE_TB 2
#endif
template <class RT>
void launch_base_dense(cudaStream_t s, int n0, const float* A, const RT* r, float* x, int ntile, int ks,
                       size_t pstride, int tb, bool cuda_cores) {
    const int nrb = (n0 + 63) / 64;
    if (tb <= 0) tb = ks > 1 ? MG_BASE_TB : 1;  // library choice
    if (tb >= 4 && ntile >= 4) {
        const unsigned nb = (unsigned)(nrb * ((ntile + 3) / 4) * ks);
        if (cuda_cores) pdl_launch(kb_base_cc<RT, 4, 64>, nb, 128, 0, s, n0, A, r, x, ntile, ks, pstride);
        else pdl_launch(kb_base_dense<RT, 4, 64>, nb, 128, 0, s, n0, A, r, x, ntile, ks, pstride);
    } else if (tb >= 2 && ntile >= 2) {
        const unsigned nb = (unsigned)(nrb * ((ntile + 1) / 2) * ks);
        if (cuda_cores) pdl_launch(kb_base_cc<RT, 2, 64>, nb, 128, 0, s, n0, A, r, x, ntile, ks, pstride);
        else pdl_launch(kb_base_dense<RT, 2, 64>, nb, 128, 0, s, n0, A, r, x, ntile, ks, pstride);
    } else {
        const unsigned nb = (unsigned)(nrb * ntile * ks);
        if (cuda_cores) pdl_launch(kb_base_cc<RT, 1, 64>, nb, 128, 0, s, n0, A, r, x, ntile, ks, pstride);
        else pdl_launch(kb_base_dense<RT, 1, 128>, nb, 128, 0, s, n0, A, r, x, ntile, ks, pstride);
    }
}

// coarsest level without a dense inverse, or Jacobi preconditioning: x = w D^-1 r
template <class RT, bool PC>
__global__ void __launch_bounds__(NTB) kb_jacobi(Depth D, const RT* r_base, float w, double* part) {
    phase_begin();
    double rz[VF] = {0.0, 0.0, 0.0, 0.0};
    {
        ROWS_F(D, t, rb, i) {
            RT rv[VF];
            vld<RT, VF>(tv(r_base, D.n, t) + i * G + c0, rv);
            float di[VF];
            dinv_of<PC>(D, t, i, c0, di);
            float xo[VF];
#pragma unroll
            for (int e = 0; e < VF; ++e) {
                xo[e] = w * di[e] * (float)rv[e];
                rz[e] += (double)rv[e] * (double)xo[e];
            }
            vst<float, VF>(tv(D.x, D.n, t) + i * G + c0, xo);
        }
    }
    if (part) block_partial<VF>(rz, part);
}


// Coarsest level with per-column operators: x = A_c^-1 r by the column's banded
// Cholesky factor A_c = L L^T (FP32, bandwidth u).  One warp per column.  Row i of
// column c holds, at Lb[(c n + i) stride + k], L[i][i-k] for k = 1..u and 1/L[i][i]
// at k = 0; Ub holds L[i+k][i] at k >= 1.  The rows are staged through shared
// memory BAND_CHUNK at a time; the last u solution values live in a ring.
constexpr int BAND_WARPS = 4;
constexpr int BAND_CHUNK = 16;
constexpr int BAND_RING = 128;  // > largest bandwidth

template <class RT>
__global__ void __launch_bounds__(32 * BAND_WARPS) kb_base_band(int n, int u, int stride, const float* __restrict__ Lb,
                                                              const float* __restrict__ Ub, const RT* r_base,
                                                              float* x_base) {
    phase_begin();
    extern __shared__ float4 band_sm4[];
    float* band_sm = reinterpret_cast<float*>(band_sm4);
    __shared__ float ring_sm[BAND_WARPS][BAND_RING];
    __shared__ float rhs_sm[BAND_WARPS][BAND_CHUNK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gc = blockIdx.x * BAND_WARPS + warp;
    const int t = gc / G, l = gc % G;
    float* rows = band_sm + (size_t)warp * BAND_CHUNK * stride;
    float* ring = ring_sm[warp];
    float* rhs = rhs_sm[warp];
    const RT* r = r_base + (size_t)t * n * G + l;
    float* x = x_base + (size_t)t * n * G + l;
    for (int pass = 0; pass < 2; ++pass) {
        const float* F = (pass == 0 ? Lb : Ub) + (size_t)gc * n * stride;
        const int nchunk = (n + BAND_CHUNK - 1) / BAND_CHUNK;
        for (int ch = 0; ch < nchunk; ++ch) {
            // forward: chunks in increasing row order; backward: decreasing
            const int c = pass == 0 ? ch : nchunk - 1 - ch;
            const int i0 = c * BAND_CHUNK, nr = min(BAND_CHUNK, n - i0);
            __syncwarp();
            const float4* src = reinterpret_cast<const float4*>(F + (size_t)i0 * stride);
            float4* dst = reinterpret_cast<float4*>(rows);
            for (int q = lane; q < nr * stride / 4; q += 32) dst[q] = __ldg(src + q);
            if (lane < nr) rhs[lane] = pass == 0 ? (float)r[(size_t)(i0 + lane) * G] : x[(size_t)(i0 + lane) * G];
            __syncwarp();
            for (int qq = 0; qq < nr; ++qq) {
                const int q = pass == 0 ? qq : nr - 1 - qq;
                const int i = i0 + q;
                const float* row = rows + q * stride;
                float acc = 0.0f;
                for (int k = 1 + lane; k <= u; k += 32) {
                    const int j = pass == 0 ? i - k : i + k;
                    if (j >= 0 && j < n) acc += row[k] * ring[j & (BAND_RING - 1)];
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                const float v = (rhs[q] - acc) * row[0];
                if (lane == 0) {
                    ring[i & (BAND_RING - 1)] = v;
                    x[(size_t)i * G] = v;
                }
                __syncwarp();
            }
        }
    }
}

// PCG start of a Newton correction J delta = -R: columns in Newton state 1 start
// from delta = 0 with r = -R; all other columns get r = 0 and stay inactive.
__global__ void __launch_bounds__(NTB) kb_init_pc(Depth D, const double* __restrict__ R, const int* __restrict__ state,
                                                  double* x64, double* r64, double* p64, double* q64, float* z,
                                                  double* part_bb, double* part_rr, float* r32s) {
    phase_begin();
    int t, rb;
    tile_rb(D.nrb, t, rb);
    const int lc = threadIdx.x % G, gc = t * G + lc;
    const bool on = state[gc] == 1;
    double rr[1] = {0.0};
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    for (int i = rb * D.rbs + threadIdx.x / G; i < i1; i += NTB / G) {
        const size_t o = ((size_t)t * D.n + i) * G + lc;
        const double ri = on ? -R[o] : 0.0;
        x64[o] = 0.0;
        z[o] = 0.0f;
        r64[o] = ri;
        r32s[o] = (float)ri;
        p64[o] = 0.0;
        q64[o] = 0.0;
        rr[0] += ri * ri;
    }
    block_partial<1>(rr, part_bb);
    __syncthreads();
    block_partial<1>(rr, part_rr);
}

// ---------------------------------------------------------------- PCG update phases

template <class T>
struct VecOf {
    static constexpr int V = std::is_same<T, double>::value ? 2 : 4;
};

// p = z + beta p, q = L z + beta q, partial (p, q).  The FP64 form on a shared
// operator is bound by GB300's FP64 pipe; 4 resident blocks per SM (64 registers)
// keep more FP64 instructions in flight than the 3 that 76 registers allowed.
// Per-column operators (several values per entry and lane) keep the 3 (FP64) or 2
// (FP32, four values) blocks their registers allowed without a bound.
#ifndef MG_MINB_A
#define MG_MINB_A 4
#endif
template <class T, bool PC>
__host__ __device__ constexpr int minb_a() {
    return PC ? (std::is_same<T, double>::value ? 3 : 2) : MG_MINB_A;
}

// Double-float operator product acc[e] = sum_w L[w, i] z[col[w, i]][c0 + e] for an
// FP64 operator given as L = Lh + Ll (two FP32 arrays) and an FP32 vector z, in
// FP32 arithmetic: each Lh z is formed exactly as a rounded product and its FMA
// error term, the rounded products are summed by two-sum (the rounding error of
// every addition is kept), the error terms and the Ll z products are summed in
// FP32, and the two sums are widened and added once in FP64.  The result carries
// about 2^-46 of sum_j |L_ij z_j| (FP64 arithmetic: about 2^-50); it replaces 7
// FP64 FMAs per row by about 70 FP32 operations and one FP64 addition, which on
// GB300 (FP32 rate many times the FP64 rate) is the cheaper way to FP64-class
// products.
template <int V>
__device__ __forceinline__ void ell_vec_df(const int32_t* __restrict__ col, const float* __restrict__ Lh,
                                           const float* __restrict__ Ll, int n, int W, int i, const float* z, int c0,
                                           double (&acc)[V]) {
    DfAcc d[V];
    auto add = [&](float ah, float al, const float (&zv)[V]) {
#pragma unroll
        for (int e = 0; e < V; ++e) d[e].add(ah, al, zv[e]);
    };
    int32_t j[WMAX];
    float ah[WMAX], al[WMAX];
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < W) {
            j[w] = __ldg(col + w * n + i);
            ah[w] = __ldg(Lh + w * n + i);
            al[w] = __ldg(Ll + w * n + i);
        }
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < W) {
            float zv[V];
            vld<float, V>(z + j[w] * G + c0, zv);
            add(ah[w], al[w], zv);
        }
    for (int w = WMAX; w < W; ++w) {
        float zv[V];
        vld<float, V>(z + __ldg(col + w * n + i) * G + c0, zv);
        add(__ldg(Lh + w * n + i), __ldg(Ll + w * n + i), zv);
    }
#pragma unroll
    for (int e = 0; e < V; ++e) acc[e] = d[e].value();
}

template <class T, bool PC, bool DF = false>
__global__ void __launch_bounds__(NTB, minb_a<T, PC>()) kb_pcg_a(Depth D, const T* Lv, T* p_base, T* q_base, const double* beta,
                                                double* part, const CallArgs* __restrict__ ca) {
    static_assert(!DF || (std::is_same<T, double>::value && !PC), "double-float products: FP64 form, shared operator");
    phase_begin();
    constexpr int V = VecOf<T>::V, TPR = G / V, RPP = NTB / TPR;
    constexpr bool kDf = std::is_same<T, double>::value && !PC;
    if constexpr (kDf) {
        if (use_df(D, ca) != DF) return;  // the other variant runs this call
    }
    int t, rb;
    tile_rb(D.nrb, t, rb);
    if (!tile_on(D.tact, t)) return;
    const int c0 = (threadIdx.x % TPR) * V;
    T pq[V] = {};  // FP32 vectors: per-thread FP32 sums over a few rows, widened once
    T bt[V];
#pragma unroll
    for (int e = 0; e < V; ++e) bt[e] = (T)beta[t * G + c0 + e];
    const float* z = tv((const float*)D.x, D.n, t);
    T* p = tv(p_base, D.n, t);
    T* q = tv(q_base, D.n, t);
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    for (int i = rb * D.rbs + threadIdx.x / TPR; i < i1; i += RPP) {
        T lz[V], pv[V], qv[V];
        float zv[V];
        if constexpr (DF) ell_vec_df<V>(D.col, D.L32, D.Llo32, D.n, D.W, i, z, c0, lz);
        else ell_vec_w<V, T, T, float, PC>(D.col, tile_vals<PC>(Lv, D, t), D.n, D.W, i, z, c0, lz);
        vld<float, V>(z + i * G + c0, zv);
        vld<T, V>(p + i * G + c0, pv);
        vld<T, V>(q + i * G + c0, qv);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            pv[e] = widen<T, float>(zv[e]) + bt[e] * pv[e];
            qv[e] = lz[e] + bt[e] * qv[e];
            pq[e] += pv[e] * qv[e];
        }
        vst<T, V>(p + i * G + c0, pv);
        vst<T, V>(q + i * G + c0, qv);
    }
    double pqd[V];
#pragma unroll
    for (int e = 0; e < V; ++e) pqd[e] = widen<double, T>(pq[e]);
    block_partial<V>(pqd, part);
}

// d += alpha p, r -= alpha q, partial (r, r); FP64 form: also r32 = (float) r for the V-cycle
template <class T>
__global__ void __launch_bounds__(NTB) kb_pcg_b(Depth D, T* d_base, T* r_base, const T* p_base, const T* q_base,
                                                const double* alpha, double* part, float* r32_base) {
    phase_begin();
    constexpr int V = VecOf<T>::V, TPR = G / V, RPP = NTB / TPR;
    int t, rb;
    tile_rb(D.nrb, t, rb);
    if (!tile_on(D.tact, t)) return;
    const int c0 = (threadIdx.x % TPR) * V;
    T rr[V] = {};  // FP32 vectors: per-thread FP32 sums over a few rows, widened once
    T al[V];
#pragma unroll
    for (int e = 0; e < V; ++e) al[e] = (T)alpha[t * G + c0 + e];
    T* d = tv(d_base, D.n, t);
    T* r = tv(r_base, D.n, t);
    const T* p = tv(p_base, D.n, t);
    const T* q = tv(q_base, D.n, t);
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    for (int i = rb * D.rbs + threadIdx.x / TPR; i < i1; i += RPP) {
        T dv[V], rv[V], pv[V], qv[V];
        vld<T, V>(d + i * G + c0, dv);
        vld<T, V>(r + i * G + c0, rv);
        vld<T, V>(p + i * G + c0, pv);
        vld<T, V>(q + i * G + c0, qv);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            dv[e] += al[e] * pv[e];
            rv[e] -= al[e] * qv[e];
            rr[e] += rv[e] * rv[e];
        }
        vst<T, V>(d + i * G + c0, dv);
        vst<T, V>(r + i * G + c0, rv);
        if (r32_base) {
            float rf[V];
#pragma unroll
            for (int e = 0; e < V; ++e) rf[e] = (float)rv[e];
            vst<float, V>(tv(r32_base, D.n, t) + i * G + c0, rf);
        }
    }
    double rrd[V];
#pragma unroll
    for (int e = 0; e < V; ++e) rrd[e] = widen<double, T>(rr[e]);
    block_partial<V>(rrd, part);
}

// FP32+refinement, FP64 residual of the columns due for an update:
// r = b - L64 (x + d) into r32, partials ||r||^2 and S^2 = || |b| + |L| |x + d| ||^2.
// Tiles without such a column return at once.
__global__ void __launch_bounds__(NTB) kb_ru_r(Depth D, const double* b64, const double* x64, const float* d32,
                                               float* r32, const int* upd, double* part, double* part_ss) {
    phase_begin();
    int t, rb;
    tile_rb(D.nrb, t, rb);
    __shared__ int tile_any;
    if (threadIdx.x == 0) {
        int a = 0;
        for (int l = 0; l < G; ++l) a |= upd[t * G + l];
        tile_any = a;
    }
    __syncthreads();
    if (!tile_any) return;
    const int lc = threadIdx.x % G, gc = t * G + lc;
    const bool on = upd[gc] != 0;
    double rr[1] = {0.0}, ss[1] = {0.0};
    const double* x = tv(x64, D.n, t);
    const float* d = tv(d32, D.n, t);
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    for (int i = rb * D.rbs + threadIdx.x / G; i < i1; i += NTB / G) {
        if (!on) continue;
        double lx = 0.0;
        float alx = 0.0f;
        for (int w = 0; w < D.W; ++w) {
            const int64_t j = __ldg(D.col + w * D.n + i);
            const double xj = x[j * G + lc] + f2d_int(d[j * G + lc]);
            lx += __ldg(D.L64 + w * D.n + i) * xj;
            alx += fabsf(__ldg(D.L32 + w * D.n + i)) * abs_to_float(xj);
        }
        const size_t o = ((size_t)t * D.n + i) * G + lc;
        const double bi = b64[o];
        const double ri = bi - lx;
        r32[o] = (float)ri;
        rr[0] += ri * ri;
        const float si = abs_to_float(bi) + alx;
        ss[0] += (double)(si * si);
    }
    block_partial<1>(rr, part);
    __syncthreads();
    block_partial<1>(ss, part_ss);
}

// FP32+refinement: fold the FP32 correction of the updated columns into x (x += d, d = 0).
__global__ void __launch_bounds__(NTB) kb_ru_x(Depth D, double* x64, float* d32, const int* upd) {
    phase_begin();
    int t, rb;
    tile_rb(D.nrb, t, rb);
    const int lc = threadIdx.x % G, gc = t * G + lc;
    if (!upd[gc]) return;
    const int i1 = min(D.n, (rb + 1) * D.rbs);
    for (int i = rb * D.rbs + threadIdx.x / G; i < i1; i += NTB / G) {
        const size_t o = ((size_t)t * D.n + i) * G + lc;
        x64[o] += f2d_int(d32[o]);
        d32[o] = 0.0f;
    }
}

}  // namespace

// ---------------------------------------------------------------- plan: buffers + graph
struct GraphPlan {
    const StepOp* op = nullptr;
    int ntile = 0, precision = 0, precond = 1, nu = 2;
    bool pc = false;   // per-column operators (Newton Jacobians), see graph_plan_pc
    int rbs0 = 0, rbs1 = 0, base_tb = 0;  // launch shape (0: library choice)
    int hf = 0;                            // mg_solver_opts::halo_fusion
    int bc = 0;                            // mg_solver_opts::base_cores
    bool base_cc = false;                  // dense base solve on the CUDA cores
    PcOperator pco{};
    float omega = 0.7f;
    int smoother = 0;
    double cheb_ratio = 0.0;
    float wsm[MG_MAX_DEPTH][MG_MAX_NU] = {};  // sweep weights of each depth's pre-smoothing
    bool wlam = false;  // per-column operators with Chebyshev weights: divide by pco.lam[d]
    std::vector<DBuf> bufs;
    DBuf args, cols, part;
    std::vector<Depth> depth;
    Cols st{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr, cap2 = nullptr;
    double *x64 = nullptr, *r64 = nullptr, *p64 = nullptr, *q64 = nullptr, *b64 = nullptr;
    float *d32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    float* r32s = nullptr;  // FP64 form: FP32 shadow of the residual
    float* split = nullptr; // FP64 form, shared operator: x_prev and guess as FP32 parts (kb_split)
    ~GraphPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        if (cap2) cudaStreamDestroy(cap2);
    }
};

void graph_plan_delete(GraphPlan* p) { delete p; }

namespace {

void* alloc(GraphPlan& P, size_t bytes) {
    P.bufs.emplace_back();
    P.bufs.back().ensure(bytes);
    return P.bufs.back().p;
}

inline unsigned grid(int ntile, int nrb) { return (unsigned)(ntile * nrb); }


// shared memory of kb_smooth2 (s1 on R + 2H rows; staged: also s0 on R + 4H rows)
inline size_t smooth2_smem(int R, int H, int cw, bool stage) {
    return (size_t)((R + 2 * H) + (stage ? R + 4 * H : 0)) * cw * sizeof(float);
}

template <bool FIRST>
void smooth2_launch(GraphPlan& P, const Depth& D, cudaStream_t s, const float* src, float* dst, float wa, float wb) {
    const unsigned g = (unsigned)(P.ntile * (G / D.f_cw) * D.f_nrb);
    const size_t smem = smooth2_smem(D.f_R, D.f_H, D.f_cw, D.f_stage);
    if (D.f_stage) {
        if (D.f_cw == 8) pdl_launch(kb_smooth2<8, FIRST, true>, g, NT2, smem, s, D, src, dst, wa, wb);
        else pdl_launch(kb_smooth2<16, FIRST, true>, g, NT2, smem, s, D, src, dst, wa, wb);
    } else {
        if (D.f_cw == 8) pdl_launch(kb_smooth2<8, FIRST, false>, g, NT2, smem, s, D, src, dst, wa, wb);
        else pdl_launch(kb_smooth2<16, FIRST, false>, g, NT2, smem, s, D, src, dst, wa, wb);
    }
}

void prolong_res_launch(GraphPlan& P, const Depth& D, const Depth& C, cudaStream_t s, int parts, size_t pstride,
                        float* sv) {
    const unsigned g = (unsigned)(P.ntile * (G / D.f_cw) * D.f_nrb);
    const size_t smem = smooth2_smem(D.f_R, D.f_H, D.f_cw, false);
    if (D.f_cw == 8) pdl_launch(kb_prolong_res<8>, g, NT2, smem, s, D, C, parts, pstride, sv);
    else pdl_launch(kb_prolong_res<16>, g, NT2, smem, s, D, C, parts, pstride, sv);
}

// one preconditioner application on the capture stream: z = B r into depth[0].x;
// the last kernel writes the (r, z) partials into part.  PC: per-column operators
// at every depth and a per-column banded Cholesky factor on the base depth.
template <class RT, bool PC>
void capture_precondition_t(GraphPlan& P, cudaStream_t s, const RT* rtop, double* part) {
    const int nd = (int)P.depth.size();
    const float w = P.omega;  // base-depth Jacobi sweep without a dense inverse
    if (P.precond == 0) {
        Depth& D = P.depth[0];
        pdl_launch(kb_jacobi<RT, PC>, grid(P.ntile, D.nrb), NTB, 0, s, D, rtop, 1.0f, part);
        return;
    }
    std::vector<int> sel(nd, 0);
    for (int d = 0; d < nd - 1; ++d) {
        Depth& D = P.depth[d];
        const float* ws = P.wsm[d];
        const unsigned* lam = P.wlam ? P.pco.lam + d : nullptr;
        int sw;
        if (!PC && std::is_same<RT, float>::value && D.f_cw && P.nu >= 2) {
            // sweeps 0 and 1 in one launch: x from the residual, s into sa
            smooth2_launch<true>(P, D, s, d == 0 ? (const float*)rtop : D.r, D.sa, ws[0], ws[1]);
            sw = 2;
        } else {
            if (d == 0) pdl_launch(kb_smooth_first<RT, PC>, grid(P.ntile, D.nrb), NTB, 0, s, D, rtop, ws[0], lam);
            else pdl_launch(kb_smooth_first<float, PC>, grid(P.ntile, D.nrb), NTB, 0, s, D, D.r, ws[0], lam);
            sw = 1;
        }
        int sl = 0;
        while (sw < P.nu) {
            if (!PC && D.f_cw && sw + 1 < P.nu) {
                smooth2_launch<false>(P, D, s, sl ? D.sb : D.sa, sl ? D.sa : D.sb, ws[sw], ws[sw + 1]);
                sw += 2;
            } else {
                pdl_launch(kb_smooth<RT, PC>, grid(P.ntile, D.nrb), NTB, 0, s, D, sl ? D.sb : D.sa, sl ? D.sa : D.sb,
                           nullptr, ws[sw], lam, nullptr);
                sw += 1;
            }
            sl ^= 1;
        }
        sel[d] = sl;
        Depth& C = P.depth[d + 1];
        pdl_launch(kb_restrict, grid(P.ntile, C.nrb), NTB, 0, s, D, C, sl ? D.sb : D.sa);
    }
    Depth& B = P.depth[nd - 1];
    const size_t pstride = (size_t)P.ntile * B.n * G;
    const int ks = nd == 1 ? 1 : BASE_KSPLIT;
    int parts = 1;
    if (PC) {
        const unsigned nb = (unsigned)(P.ntile * G / BAND_WARPS);
        const size_t smem = (size_t)BAND_WARPS * BAND_CHUNK * P.pco.band_stride * sizeof(float);
        if (nd == 1) pdl_launch(kb_base_band<RT>, nb, 32 * BAND_WARPS, smem, s, B.n, P.pco.band_u, P.pco.band_stride,
                                                                       P.pco.band_L, P.pco.band_U, rtop, B.x);
        else pdl_launch(kb_base_band<float>, nb, 32 * BAND_WARPS, smem, s, B.n, P.pco.band_u, P.pco.band_stride,
                                                                  P.pco.band_L, P.pco.band_U, B.r, B.x);
    } else if (P.op->base_inv.p) {
        if (nd == 1)
            launch_base_dense<RT>(s, B.n, P.op->base_inv.as<float>(), rtop, B.x, P.ntile, 1, 0, P.base_tb, P.base_cc);
        else
            launch_base_dense<float>(s, B.n, P.op->base_inv.as<float>(), B.r, B.x, P.ntile, ks, pstride, P.base_tb,
                                     P.base_cc);
        parts = ks;
    } else {
        if (nd == 1) pdl_launch(kb_jacobi<RT, PC>, grid(P.ntile, B.nrb), NTB, 0, s, B, rtop, w, nullptr);
        else pdl_launch(kb_jacobi<float, PC>, grid(P.ntile, B.nrb), NTB, 0, s, B, B.r, w, nullptr);
    }
    if (nd == 1) {
        // z is final; a zero-weight sweep accumulates (r, z) for a single-level hierarchy
        Depth& D = P.depth[0];
        pdl_launch(kb_smooth<RT, PC>, grid(P.ntile, D.nrb), NTB, 0, s, D, D.x, nullptr, rtop, 0.0f,
                   (const unsigned*)nullptr, part);
        return;
    }
    for (int d = nd - 2; d >= 0; --d) {
        Depth& D = P.depth[d];
        Depth& C = P.depth[d + 1];
        const bool from_base = d + 1 == nd - 1;
        int sl = sel[d];
        if (!PC && D.f_cw) {
            prolong_res_launch(P, D, C, s, from_base ? parts : 1, pstride, sl ? D.sb : D.sa);
        } else {
            pdl_launch(kb_prolong, grid(P.ntile, D.nrb), NTB, 0, s, D, C, from_base ? parts : 1, pstride);
            pdl_launch(kb_resupdate<PC>, grid(P.ntile, D.nrb), NTB, 0, s, D, sl ? D.sb : D.sa);
        }
        for (int sw = 0; sw < P.nu;) {
            // a pair of sweeps in one launch unless its second sweep is the finest
            // depth's last, which also accumulates (r, z)
            const bool pair_last = sw + 1 == P.nu - 1;
            if (!PC && D.f_cw && sw + 1 < P.nu && !(pair_last && d == 0)) {
                smooth2_launch<false>(P, D, s, sl ? D.sb : D.sa, pair_last ? nullptr : (sl ? D.sa : D.sb),
                                      P.wsm[d][P.nu - 1 - sw], P.wsm[d][P.nu - 2 - sw]);
                sw += 2;
                sl ^= 1;
                continue;
            }
            const bool last = sw == P.nu - 1;
            const bool top = last && d == 0;
            pdl_launch(kb_smooth<RT, PC>, grid(P.ntile, D.nrb), NTB, 0, s, D, sl ? D.sb : D.sa,
                       last ? nullptr : (sl ? D.sa : D.sb), top ? rtop : nullptr, P.wsm[d][P.nu - 1 - sw],
                       P.wlam ? P.pco.lam + d : nullptr, top ? part : nullptr);
            sl ^= 1;
            ++sw;
        }
    }
}

template <class RT>
void capture_precondition(GraphPlan& P, cudaStream_t s, const RT* rtop, double* part) {
    if (P.pc) capture_precondition_t<RT, true>(P, s, rtop, part);
    else capture_precondition_t<RT, false>(P, s, rtop, part);
}

// FP32+refinement: the FP64 residual update of the columns due for one, the
// decisions taken on it (and the loop condition), then x += d for those columns
void capture_reliable_update(GraphPlan& P, cudaStream_t s, const CallArgs* ca, cudaGraphConditionalHandle h,
                             int use_cond) {
    Depth& D0 = P.depth[0];
    const size_t np = (size_t)P.ntile * D0.nrb * G;
    double* part = P.part.as<double>();
    double* part_rr = part + np;
    double* part_ss = part + 2 * np;
    pdl_launch(kb_ru_r, grid(P.ntile, D0.nrb), NTB, 0, s, D0, (const double*)P.b64, (const double*)P.x64,
               (const float*)P.d32, P.r32, (const int*)P.st.upd, part_rr, part_ss);
    pdl_launch(kb_scalar_ru, P.ntile, NTB, 0, s, P.st, (const double*)part_rr, (const double*)part_ss, D0.nrb, ca, h,
               use_cond);
    pdl_launch(kb_ru_x, grid(P.ntile, D0.nrb), NTB, 0, s, D0, P.x64, P.d32, (const int*)P.st.upd);
}

// one PCG iteration body (after the preconditioner)
template <class T>
void capture_pcg_body(GraphPlan& P, cudaStream_t s, T* d, T* r, T* p, T* q, const T* Lv, const CallArgs* ca,
                      int inner, cudaGraphConditionalHandle h, int use_cond) {
    Depth& D0 = P.depth[0];
    double* part = P.part.as<double>();
    // the V-cycle always reads an FP32 residual: the FP64 form keeps an FP32 shadow of r
    float* rf = nullptr;
    if constexpr (std::is_same<T, double>::value) rf = P.r32s;
    else rf = r;
    capture_precondition<float>(P, s, rf, part);
    pdl_launch(kb_scalar_gamma, P.ntile, NTB, 0, s, P.st, part, D0.nrb);
    if (P.pc) {
        pdl_launch(kb_pcg_a<T, true>, grid(P.ntile, D0.nrb), NTB, 0, s, D0, Lv, p, q, P.st.beta, part, ca);
    } else {
        pdl_launch(kb_pcg_a<T, false>, grid(P.ntile, D0.nrb), NTB, 0, s, D0, Lv, p, q, P.st.beta, part, ca);
        if constexpr (std::is_same<T, double>::value)
            if (D0.Llo32)
                pdl_launch(kb_pcg_a<T, false, true>, grid(P.ntile, D0.nrb), NTB, 0, s, D0, Lv, p, q, P.st.beta, part,
                           ca);
    }
    pdl_launch(kb_scalar_alpha, P.ntile, NTB, 0, s, P.st, part, D0.nrb);
    pdl_launch(kb_pcg_b<T>, grid(P.ntile, D0.nrb), NTB, 0, s, D0, d, r, p, q, P.st.alpha, part,
                                                       std::is_same<T, double>::value ? P.r32s : nullptr);
    if (inner) {
        pdl_launch(kb_scalar_conv_ru, P.ntile, NTB, 0, s, P.st, part, D0.nrb, ca);
        capture_reliable_update(P, s, ca, h, use_cond);
    } else {
        pdl_launch(kb_scalar_conv, P.ntile, NTB, 0, s, P.st, part, D0.nrb, ca, inner, h, use_cond);
    }
}

// append a WHILE node at the capture's current position; returns its body graph
cudaGraph_t add_while(cudaStream_t s, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    MG_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    MG_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm));
    MG_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return prm.conditional.phGraph_out[0];
}

cudaGraphConditionalHandle new_handle(cudaStream_t s) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    MG_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h;
    MG_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    return h;
}

// Launch shape of kb_smooth2 on a depth of n rows with bandwidth H over ntile
// column tiles: columns (8 or 16) and rows per block such that two
// blocks of NT2 threads fit an SM (shared memory smooth2_smem each) and the halo is
// at most 60 % of a block's rows (beyond that two single sweeps are cheaper); among
// those the one with the least work per SM.  The first sweep is bound by L1
// throughput (its gathers); a warp's gather costs one L1 wavefront per 128-byte
// line it touches, so a row costs the same for 8 and 16 columns (8-column blocks
// use half of each line), and the cost is waves x (halo-extended rows + half the
// block's own rows for the second sweep).  False if none qualifies.
constexpr size_t SMOOTH2_SMEM_MAX = 113 * 1024;
bool smooth2_shape(int n, int H, int ntile, int sms, bool stage, int& cw, int& R) {
    double best = 0.0;
    bool ok = false;
    for (int c : {16, 8})  // ties go to 16 columns: half the blocks for the same time
        for (int r : {2048, 1536, 1024, 768, 512, 384, 256}) {
            if (2.0 * H > 0.6 * r || smooth2_smem(r, H, c, stage) > SMOOTH2_SMEM_MAX) continue;
            const long blocks = (long)ntile * (G / c) * ((n + r - 1) / r);
            const long waves = (blocks + 2L * sms - 1) / (2L * sms);
            const double cost = (double)waves * (std::min(n, r + 2 * H) + 0.5 * std::min(n, r));
            if (!ok || cost < best) {
                ok = true;
                best = cost;
                cw = c;
                R = r;
            }
        }
    return ok;
}

template <int CW, bool FIRST, bool STAGE>
void smooth2_allow_smem() {
    MG_CUDA(cudaFuncSetAttribute(kb_smooth2<CW, FIRST, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMOOTH2_SMEM_MAX));
}

// The FP64 form's set-up phase: with split buffers, kb_split and both variants of
// kb_init (the one this call's tolerance selects runs, the others return at once).
void launch_init0(GraphPlan& P, cudaStream_t s, const CallArgs* ca, double inv_dt, const double* F, double J0,
                  double* part, double* part2, double* part3) {
    Depth& D0 = P.depth[0];
    const unsigned g = grid(P.ntile, D0.nrb);
    const size_t e0 = (size_t)P.ntile * D0.n * G;
    float* sp = P.split;
    if (sp && D0.M32) kb_split<<<g, NTB, 0, s>>>(D0, ca, sp, sp + e0, sp + 2 * e0, sp + 3 * e0);
    kb_init<0><<<g, NTB, 0, s>>>(D0, ca, inv_dt, F, J0, P.x64, P.r64, P.p64, P.q64, nullptr, D0.x, part, part2, part3,
                                 P.r32s, nullptr, nullptr, nullptr, sp && D0.M32 ? sp : nullptr);
    if (sp && D0.M32)
        kb_init<0, true><<<g, NTB, 0, s>>>(D0, ca, inv_dt, F, J0, P.x64, P.r64, P.p64, P.q64, nullptr, D0.x, part,
                                           part2, part3, P.r32s, nullptr, nullptr, nullptr, sp);
}

GraphPlan* build_plan(mg_ctx* c, const StepOp& op, int ntile, const mg_solver_opts& so,
                      const PcOperator* pco = nullptr) {
    auto* P = new GraphPlan();
    try {
        P->op = &op;
        P->ntile = ntile;
        P->rbs0 = so.rows_per_block;
        P->rbs1 = so.coarse_rows_per_block;
        P->base_tb = so.base_tiles;
        P->hf = so.halo_fusion;
        P->bc = so.base_cores;
        P->base_cc = so.base_cores != MG_BASE_TENSOR;
        if (pco) {
            P->pc = true;
            P->pco = *pco;
        }
        P->precision = so.precision;
        P->precond = so.precond;
        P->nu = smooth_sweeps(so);
        P->omega = so.omega > 0.0 ? (float)so.omega : 0.7f;
        P->smoother = so.smoother;
        P->cheb_ratio = so.cheb_ratio;
        // per-column Jacobians: weights for a unit bound, divided on the device by the
        // bound of the current Jacobians (damped Jacobi without one)
        P->wlam = P->pc && P->pco.lam && so.smoother == MG_SMOOTH_CHEBYSHEV;
        for (int d = 0; d < (int)op.mg.size() && d < MG_MAX_DEPTH; ++d)
            smoother_weights(P->pc ? (P->wlam ? 1.0 : 0.0) : op.mg[d]->lam, so, P->nu, P->wsm[d]);
        const MeshLevel& m0 = c->meshes[op.mesh];
        const int nd = so.precond == MG_PRECOND_MULTIGRID ? (int)op.mg.size() : 1;
        for (int d = 0; d < nd; ++d) {
            const MgDepth& md = *op.mg[d];
            const MeshLevel& mm = c->meshes[md.mesh];
            Depth D = {};
            D.n = (int)md.n;
            D.W = md.W;
            if (d > 0) D.rbs = so.coarse_rows_per_block > 0 ? so.coarse_rows_per_block : MG_RBS1;
            else D.rbs = so.rows_per_block > 0 ? so.rows_per_block : (D.n > 8192 ? MG_RBS0_LARGE : MG_RBS0);
            D.nrb = (D.n + D.rbs - 1) / D.rbs;
            D.col = mm.ell_col.as<int32_t>();
            D.L64 = md.L64.as<double>();
            D.M64 = md.M64.as<double>();
            D.L32 = md.L32.as<float>();
            D.Llo32 = md.Llo32.as<float>();
            D.M32 = md.M32.as<float>();
            D.Mlo32 = md.Mlo32.as<float>();
            D.LD32 = md.LD32.as<float>();
            D.dinv32 = md.dinv32.as<float>();
            if (P->pc) {  // per-column Jacobians replace the step operator's values
                D.L64 = pco->d[d].J64;
                D.M64 = nullptr;
                D.L32 = pco->d[d].J32;
                D.Llo32 = nullptr;
                D.M32 = D.Mlo32 = nullptr;
                D.LD32 = pco->d[d].LD32;
                D.dinv32 = pco->d[d].dinv32;
            }
            if (d + 1 < nd) {
                D.par = mm.par.as<int32_t>();
                D.pw = mm.pw.as<float>();
                D.rt_W = mm.rt_W;
                D.rt_col = mm.rt_col.as<int32_t>();
                D.rt_w = mm.rt_w.as<float>();
            }
            const size_t e = (size_t)ntile * D.n * G;
            const bool base_split =
                !P->pc && so.precond == MG_PRECOND_MULTIGRID && d == nd - 1 && nd > 1 && op.base_inv.p;
            D.x = (float*)alloc(*P, e * 4 * (base_split ? BASE_KSPLIT : 1));
            if (so.precond == MG_PRECOND_MULTIGRID && d + 1 < nd) {
                D.sa = (float*)alloc(*P, e * 4);
                D.sb = (float*)alloc(*P, e * 4);
                D.y = (float*)alloc(*P, e * 4);
            }
            if (d > 0) D.r = (float*)alloc(*P, e * 4);
            // halo-fused kernels (two sweeps per launch, prolongation with residual
            // update) on smoothed depths of shared operators
            const bool stage = so.halo_fusion == 3;
            if (!P->pc && so.precond == MG_PRECOND_MULTIGRID && d + 1 < nd && so.halo_fusion != 1 &&
                smooth2_shape(D.n, mm.ell_bw, ntile, c->sm_count > 0 ? c->sm_count : 1, stage, D.f_cw, D.f_R)) {
                D.f_H = mm.ell_bw;
                D.f_nrb = (D.n + D.f_R - 1) / D.f_R;
                D.f_stage = stage;
                smooth2_allow_smem<8, true, false>();
                smooth2_allow_smem<8, false, false>();
                smooth2_allow_smem<16, true, false>();
                smooth2_allow_smem<16, false, false>();
                smooth2_allow_smem<8, true, true>();
                smooth2_allow_smem<8, false, true>();
                smooth2_allow_smem<16, true, true>();
                smooth2_allow_smem<16, false, true>();
                MG_CUDA(cudaFuncSetAttribute(kb_prolong_res<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SMOOTH2_SMEM_MAX));
                MG_CUDA(cudaFuncSetAttribute(kb_prolong_res<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SMOOTH2_SMEM_MAX));
            }
            P->depth.push_back(D);
        }
        const size_t e0 = (size_t)ntile * m0.n * G;
        P->x64 = (double*)alloc(*P, e0 * 8);
        if (so.precision == MG_FP64) {
            P->r64 = (double*)alloc(*P, e0 * 8);
            P->p64 = (double*)alloc(*P, e0 * 8);
            P->q64 = (double*)alloc(*P, e0 * 8);
            P->r32s = (float*)alloc(*P, e0 * 4);
            if (!P->pc) P->split = (float*)alloc(*P, e0 * 4 * 4);
        } else {
            P->b64 = (double*)alloc(*P, e0 * 8);
            P->d32 = (float*)alloc(*P, e0 * 4);
            P->r32 = (float*)alloc(*P, e0 * 4);
            P->p32 = (float*)alloc(*P, e0 * 4);
            P->q32 = (float*)alloc(*P, e0 * 4);
        }
        const int kpad = ntile * G;
        P->cols.ensure((size_t)kpad * (7 * sizeof(double) + 8 * sizeof(int)) + (size_t)ntile * sizeof(int) + 64);
        char* cb = (char*)P->cols.p;
        P->st.bb = (double*)cb;
        P->st.gam = P->st.bb + kpad;
        P->st.beta = P->st.gam + kpad;
        P->st.alpha = P->st.beta + kpad;
        P->st.ref = P->st.alpha + kpad;
        P->st.prev = P->st.ref + kpad;
        P->st.ss = P->st.prev + kpad;
        P->st.act = (int*)(P->st.ss + kpad);
        P->st.outer = P->st.act + kpad;
        P->st.iters = P->st.outer + kpad;
        P->st.bad = P->st.iters + kpad;
        P->st.upd = P->st.bad + kpad;
        P->st.nup = P->st.upd + kpad;
        P->st.stall = P->st.nup + kpad;
        P->st.lastu = P->st.stall + kpad;
        P->st.ctr = P->st.lastu + kpad;
        P->st.tact = P->st.ctr + 16;  // after the 4 counters (padded)
        for (auto& d : P->depth) d.tact = P->st.tact;
        const int nrb0 = P->depth[0].nrb;
        P->part.ensure((size_t)3 * ntile * std::max(nrb0, 1) * G * sizeof(double));
        P->args.ensure(sizeof(CallArgs));
        // ---- capture
        MG_CUDA(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
        MG_CUDA(cudaStreamCreateWithFlags(&P->cap2, cudaStreamNonBlocking));
        MG_CUDA(cudaGraphCreate(&P->graph, 0));
        cudaStream_t s = P->cap;
        MG_CUDA(cudaStreamBeginCaptureToGraph(s, P->graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        const CallArgs* ca = P->args.as<CallArgs>();
        Depth& D0 = P->depth[0];
        double* part = P->part.as<double>();
        double* part2 = part + (size_t)ntile * nrb0 * G;
        double* part3 = part2 + (size_t)ntile * nrb0 * G;
        const double inv_dt = 1.0 / op.dt;
        const double J0 = c->pwm.J0;
        if (so.precision == MG_FP64) {
            cudaGraphConditionalHandle h = new_handle(s);
            if (P->pc)
                kb_init_pc<<<grid(ntile, nrb0), NTB, 0, s>>>(D0, pco->R, pco->state, P->x64, P->r64, P->p64, P->q64,
                                                             D0.x, part, part2, P->r32s);
            else
                launch_init0(*P, s, ca, inv_dt, m0.F.as<double>(), J0, part, part2, part3);
            kb_scalar_init0<<<1, NSB, 0, s>>>(P->st, part, part2, P->pc ? nullptr : part3, nrb0, kpad, ca, h, 1);
            cudaGraph_t body = add_while(s, h);
            if (!P->pc) kb_final<<<grid(ntile, nrb0), NTB, 0, s>>>(D0, ca, P->x64, nullptr);
            kb_scalar_final<<<1, NSB, 0, s>>>(P->st, kpad, ca, 0, (unsigned long long*)c->counters.p,
                                              (int*)((char*)c->counters.p + 8));
            MG_CUDA(cudaStreamEndCapture(s, &P->graph));
            MG_CUDA(cudaStreamBeginCaptureToGraph(P->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            capture_pcg_body<double>(*P, P->cap2, P->x64, P->r64, P->p64, P->q64, D0.L64, ca, 0, h, 1);
            MG_CUDA(cudaStreamEndCapture(P->cap2, &body));
        } else {
            // FP32 PCG with reliable updates: the FP32 recurrence runs on; a column whose
            // FP32 residual has fallen by inner_tol since its last FP64 residual gets
            // x += d and its residual replaced by b - L64 x (FP64), then continues
            cudaGraphConditionalHandle h = new_handle(s);
            kb_init<1><<<grid(ntile, nrb0), NTB, 0, s>>>(D0, ca, inv_dt, m0.F.as<double>(), J0, P->x64, nullptr,
                                                         nullptr, nullptr, P->b64, D0.x, part, part2, nullptr,
                                                         nullptr, P->d32, P->p32, P->q32);
            kb_scalar_init1<<<1, NSB, 0, s>>>(P->st, part, nrb0, kpad, ca);
            capture_reliable_update(*P, s, ca, h, 1);
            cudaGraph_t body = add_while(s, h);
            kb_final<<<grid(ntile, nrb0), NTB, 0, s>>>(D0, ca, P->x64, P->d32);
            kb_scalar_final<<<1, NSB, 0, s>>>(P->st, kpad, ca, 1, (unsigned long long*)c->counters.p,
                                              (int*)((char*)c->counters.p + 8));
            MG_CUDA(cudaStreamEndCapture(s, &P->graph));
            MG_CUDA(cudaStreamBeginCaptureToGraph(P->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            capture_pcg_body<float>(*P, P->cap2, P->d32, P->r32, P->p32, P->q32, D0.L32, ca, 1, h, 1);
            MG_CUDA(cudaStreamEndCapture(P->cap2, &body));
        }
        MG_CUDA(cudaGraphInstantiate(&P->exec, P->graph, 0));
        return P;
    } catch (...) {
        cudaStreamCaptureStatus cs;
        for (cudaStream_t s : {P->cap, P->cap2})
            if (s && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t junk = nullptr;
                cudaStreamEndCapture(s, &junk);
                if (junk && junk != P->graph) cudaGraphDestroy(junk);
            }
        cudaGetLastError();
        delete P;
        throw;
    }
}

}  // namespace

// Profiling aid: the kernels of the graph path launched directly on the stream for
// a fixed number of PCG iterations (no graph, no early exit), so that per-kernel
// profilers can see every launch.  Selected by MGRIT_EM_EAGER=<iterations>.
static void run_eager(mg_ctx* c, GraphPlan& P, int iters) {
    cudaStream_t s = c->stream;
    const MeshLevel& m0 = c->meshes[P.op->mesh];
    Depth& D0 = P.depth[0];
    const int nrb0 = D0.nrb, kpad = P.ntile * G;
    double* part = P.part.as<double>();
    double* part2 = part + (size_t)P.ntile * nrb0 * G;
    double* part3 = part2 + (size_t)P.ntile * nrb0 * G;
    const CallArgs* ca = P.args.as<CallArgs>();
    if (P.precision == MG_FP64) {
        launch_init0(P, s, ca, 1.0 / P.op->dt, m0.F.as<double>(), c->pwm.J0, part, part2, part3);
        kb_scalar_init0<<<1, NSB, 0, s>>>(P.st, part, part2, part3, nrb0, kpad, ca, 0, 0);
        for (int it = 0; it < iters; ++it)
            capture_pcg_body<double>(P, s, P.x64, P.r64, P.p64, P.q64, D0.L64, ca, 0, 0, 0);
        kb_final<<<grid(P.ntile, nrb0), NTB, 0, s>>>(D0, ca, P.x64, nullptr);
    } else {
        kb_init<1><<<grid(P.ntile, nrb0), NTB, 0, s>>>(D0, ca, 1.0 / P.op->dt, m0.F.as<double>(), c->pwm.J0, P.x64,
                                                       nullptr, nullptr, nullptr, P.b64, D0.x, part, part2, nullptr,
                                                       nullptr, P.d32, P.p32, P.q32);
        kb_scalar_init1<<<1, NSB, 0, s>>>(P.st, part, nrb0, kpad, ca);
        capture_reliable_update(P, s, ca, 0, 0);
        for (int it = 0; it < iters; ++it)
            capture_pcg_body<float>(P, s, P.d32, P.r32, P.p32, P.q32, D0.L32, ca, 1, 0, 0);
        kb_final<<<grid(P.ntile, nrb0), NTB, 0, s>>>(D0, ca, P.x64, P.d32);
    }
    kb_scalar_final<<<1, NSB, 0, s>>>(P.st, kpad, ca, P.precision == MG_FP64 ? 0 : 1,
                                      (unsigned long long*)c->counters.p, (int*)((char*)c->counters.p + 8));
    MG_CUDA(cudaGetLastError());
}

// Batched step through the graph path.  The plan (buffers + instantiated graph) is
// built on first use for (operator, tile count, form, preconditioner) and reused.
void phi_batch_graph(mg_ctx* c, const StepOp& op, const PhiIO& io, const mg_solver_opts& so, SolveCounters* counters) {
    const int ntile = (io.k + G - 1) / G;
    GraphPlan* P = nullptr;
    for (auto* q : c->plans)
        if (!q->pc && q->op == &op && q->ntile == ntile && q->precision == so.precision && q->precond == so.precond &&
            q->nu == smooth_sweeps(so) && q->omega == (so.omega > 0.0 ? (float)so.omega : 0.7f) &&
            q->smoother == so.smoother && q->cheb_ratio == so.cheb_ratio &&
            q->rbs0 == so.rows_per_block && q->rbs1 == so.coarse_rows_per_block && q->base_tb == so.base_tiles &&
            q->hf == so.halo_fusion && q->bc == so.base_cores) {
            P = q;
            break;
        }
    if (!P) {
        c->counters.ensure(16);
        P = build_plan(c, op, ntile, so);
        c->plans.push_back(P);
    }
    CallArgs a = {};
    a.xprev = io.xprev;
    a.ld_prev = io.ld_prev;
    a.g = io.g;
    a.ld_g = io.ld_g;
    a.guess = io.guess;
    a.ld_guess = io.ld_guess;
    a.xout = io.xout;
    a.ld_out = io.ld_out;
    a.wave = io.wave;
    a.t0 = io.t0;
    a.tstride = io.tstride;
    a.k = io.k;
    const double tol = so.precision == MG_FP64 ? so.cg_tol : so.refine_tol;
    a.tol2 = tol * tol;
    a.inner_tol2 = so.inner_tol * so.inner_tol;
    a.max_it = so.max_cg;
    a.max_refine = so.max_refine;
    const double fs = residual_floor(P->depth[0].W);
    a.fl_stop2 = fs * fs;
    a.fl_acc2 = (kFloorAccept * fs) * (kFloorAccept * fs);
    MG_CUDA(cudaMemcpyAsync(P->args.p, &a, sizeof(a), cudaMemcpyHostToDevice, c->stream));
    const char* eager = getenv("MGRIT_EM_EAGER");
    if (eager) run_eager(c, *P, atoi(eager));
    else MG_CUDA(cudaGraphLaunch(P->exec, c->stream));
    if (counters) {
        counters->step_solves += io.k;
        counters->batched_steps += 1;
        counters->launches += 1;
    }
}

// ---------------------------------------------------------------- per-column systems (Newton corrections)
GraphPlan* graph_plan_pc(mg_ctx* c, const StepOp& op, int ntile, const mg_solver_opts& so, const PcOperator& pco) {
    if (so.precision != MG_FP64) mg_fail(MG_EINVAL, "Newton corrections are solved in the FP64 form");
    if (pco.band_u >= BAND_RING) mg_fail(MG_EINVAL, "base mesh bandwidth too large for the banded coarse solve");
    c->counters.ensure(16);
    return build_plan(c, op, ntile, so, &pco);
}

double* graph_plan_solution(GraphPlan* p) { return p->x64; }

void graph_plan_run(mg_ctx* c, GraphPlan* P, int k, const mg_solver_opts& so) {
    CallArgs a = {};
    a.k = k;
    a.tol2 = so.cg_tol * so.cg_tol;
    a.inner_tol2 = so.inner_tol * so.inner_tol;
    a.max_it = so.max_cg;
    a.max_refine = so.max_refine;
    MG_CUDA(cudaMemcpyAsync(P->args.p, &a, sizeof(a), cudaMemcpyHostToDevice, c->stream));
    MG_CUDA(cudaGraphLaunch(P->exec, c->stream));
}
