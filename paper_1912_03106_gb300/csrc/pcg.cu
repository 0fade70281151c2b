// Batched backward-Euler step solves: one persistent, cluster-resident launch.
//
// Each column c of a batch is one time interval (F-relaxation), one C-point
// (C-relaxation, residual) or one time step (sequential stepping) of Sec. 2.1.
// For every column the kernel solves the step of Eq. discrete_system,
//     (M/dt + K) x = (M/dt) x_prev + J0 sum_s b_s(t_c) F_s,
// then writes x + g (g = FAS right-hand side on coarse levels, Algorithm 1).
//
// Mapping onto GB300: a thread-block cluster owns a tile of KT columns; each CTA
// of the cluster owns a contiguous row range of every mesh level.  Matrices are
// ELL (column-major, width W), work vectors tile-major (tile, row, column), so the
// KT values one nonzero multiplies are one contiguous segment.  A thread handles
// V adjacent columns of a row with one vector load (float4 / double2), and every
// phase first issues the loads of two rows and only then computes and stores,
// so enough loads are in flight to cover L2 and HBM latency.  The whole solve
// runs inside the launch: dot products are reduced by warp shuffles, across
// warps in shared memory and across the cluster through distributed shared
// memory behind a cluster barrier; every CTA adds the partials of all ranks in
// the same order, so all CTAs take the same per-column decisions (convergence
// masks) and leave the loop together, and repeated runs are bitwise identical.
// Nothing on the data path uses atomics.
//
// Preconditioner: one geometric-multigrid V-cycle in FP32 over the nested mesh
// hierarchy (the hierarchy the spatial coarsening of Sec. 2.2 / Sec. 3.4 uses):
// damped-Jacobi smoothing whose residual update is fused into the same sweep,
// restriction by P^T, nodal-interpolation prolongation P, and a dense FP32
// inverse on the coarsest mesh.  Coarse operators are the re-discretised
// M/dt + K, equal to the Galerkin products P^T L P for nested P1 spaces with
// coefficients constant on coarse elements.  Jacobi is kept as an option.
//
// Two arithmetic forms:
//   FP64        PCG with FP64 vectors, operator and dot products until
//               ||b - L x|| <= cg_tol ||b|| per column (preconditioner FP32).
//   FP32+refine FP64 outer iterative refinement r = b - L64 x, inner PCG in FP32
//               with FP32 accumulation on L32 d = r, x += d, until
//               ||b - L64 x|| <= refine_tol ||b|| or the FP64 residual stalls.
// Converged columns keep running with alpha = 0 (their iterate is frozen), so
// the lanes of a tile never diverge in control flow.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "vec.cuh"

namespace cg = cooperative_groups;

namespace {

using namespace mgv;

constexpr int NT = 256;  // threads per CTA
constexpr int NWARP = NT / 32;
#ifndef MG_RB
#define MG_RB 2
#endif
#ifndef MG_MINB
#define MG_MINB 1
#endif
constexpr int RB = MG_RB;  // rows whose loads are issued together

struct DepthArgs {
    int n;
    int W;
    const int32_t* col;  // W x n
    const double* L64;
    const double* M64;
    const float* L32;
    const float* LD32;
    const double* dinv64;
    const float* dinv32;
    const int32_t* par;  // 2 x n coarse parents (transfer to depth + 1)
    const float* pw;
    int rt_W;            // P^T as ELL over depth + 1 rows
    const int32_t* rt_col;
    const float* rt_w;
    float *x, *sa, *sb, *y, *r;  // tile-major work vectors
};

struct PcgArgs {
    int nd;
    DepthArgs d[MG_MAX_DEPTH];
    const float* base_inv;  // dense inverse on the deepest level (or null)
    int precond;            // 0 Jacobi, 1 multigrid V-cycle
    int nu;                 // smoothing sweeps before and after the coarse correction
    float omega;            // Jacobi weight of the base-depth sweep without a dense inverse
    float wsm[MG_MAX_DEPTH][MG_MAX_NU];  // sweep weights of each depth's pre-smoothing
    double inv_dt;
    const double* F;  // 3 x n (depth 0)
    double J0;
    const double* wave;
    int64_t t0, tstride;
    const double* xprev;
    int64_t ld_prev;
    const double* g;
    int64_t ld_g;
    const double* guess;
    int64_t ld_guess;
    double* xout;
    int64_t ld_out;
    int k;
    double *b64, *x64, *r64, *p64, *q64;  // tile-major, depth 0
    float *d32, *r32, *p32, *q32;
    double tol;
    double inner_tol;
    double fl_stop2, fl_acc2;  // rounding floor of the FP64 residual (squared factors of S, see internal.h)
    int max_it;
    int max_refine;
    int mode;
    unsigned long long* iter_sum;
    int* worst;
};

// ---------------------------------------------------------------- per-CTA state
template <int KT>
struct Smem {
    double ws[3][NWARP][KT];
    double red[2][3][KT];
    double tot[3][KT];
    double bb[KT];
    double gam[KT];
    double beta[KT];
    double alpha[KT];
    double ref[KT];
    double prev[KT];
    double ss[KT];  // S^2 = || |b| + |L| |x| ||^2 of the rounding floor
    int act[KT];
    int outer[KT];
    int iters[KT];
    int bad[KT];  // a non-finite residual or right-hand side was seen
    int upd[KT];    // FP32+refine: FP64 residual update due
    int nup[KT];    // FP32+refine: FP64 residual updates done
    int stall[KT];  // FP32+refine: updates in a row that took less than 10 % off ||r||
    int lastu[KT];  // FP32+refine: the column's iteration count at its last FP64 update
    int any;
};

template <int KT>
struct Ctx {
    cg::cluster_group cl;
    int csize, rank, tile;
    int buf;
    __device__ Ctx() : cl(cg::this_cluster()) {
        csize = (int)cl.num_blocks();
        rank = (int)cl.block_rank();
        tile = blockIdx.x / csize;
        buf = 0;
    }
    __device__ void rows(int64_t n, int64_t& rb, int64_t& re) const {
        int64_t per = (n + csize - 1) / csize;
        rb = ::min(n, (int64_t)rank * per);
        re = ::min(n, rb + per);
    }
    template <class T>
    __device__ T* tv(T* base, int64_t n) const { return base + (size_t)tile * n * KT; }
};

// Thread -> (row offset, column group) for V columns per thread.
template <int KT, int V>
struct Lanes {
    static constexpr int TPR = KT / V;    // threads per row
    static constexpr int RPP = NT / TPR;  // rows per pass of the CTA
    static __device__ __forceinline__ int c0() { return (threadIdx.x % TPR) * V; }
    static __device__ __forceinline__ int roff() { return threadIdx.x / TPR; }
};

// Run a phase over the CTA's rows of an n-row level: loads of RB rows, then stores.
template <int KT, int V, class B>
__device__ __forceinline__ void run_rows(const Ctx<KT>& c, int64_t n, B& b) {
    int64_t rb64, re64;
    c.rows(n, rb64, re64);
    const int rb = (int)rb64, re = (int)re64;
    using Ln = Lanes<KT, V>;
    for (int base = rb + Ln::roff(); base < re; base += RB * Ln::RPP) {
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int i = base + q * Ln::RPP;
            if (i < re) b.load(q, i);
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int i = base + q * Ln::RPP;
            if (i < re) b.store(q, i);
        }
    }
}

// ---------------------------------------------------------------- cluster reduction
// Sum per-column partials v[q][e] (thread's columns c0 + e) over the cluster into s.tot.
template <int KT, int V, int NQ, class A>
__device__ __forceinline__ void cluster_sum(Ctx<KT>& c, Smem<KT>& s, A (&v)[NQ][V]) {
    using Ln = Lanes<KT, V>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int e = 0; e < V; ++e) {
            A x = v[q][e];
#pragma unroll
            for (int off = Ln::TPR; off < 32; off <<= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            v[q][e] = x;
        }
    if (lane < Ln::TPR) {
        const int c0 = lane * V;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int e = 0; e < V; ++e) s.ws[q][warp][c0 + e] = (double)v[q][e];
    }
    __syncthreads();
    if (threadIdx.x < NQ * KT) {
        int q = threadIdx.x / KT, cc = threadIdx.x % KT;
        A acc = 0;
        for (int w = 0; w < NWARP; ++w) acc += (A)s.ws[q][w][cc];
        s.red[c.buf][q][cc] = (double)acc;
    }
    c.cl.sync();  // release/acquire at cluster scope: partials and vector rows visible
    if (threadIdx.x < NQ * KT) {
        int q = threadIdx.x / KT, cc = threadIdx.x % KT;
        A acc = 0;
        for (int r = 0; r < c.csize; ++r) acc += (A)(*c.cl.map_shared_rank(&s.red[c.buf][q][cc], r));
        s.tot[q][cc] = (double)acc;
    }
    __syncthreads();
    c.buf ^= 1;
}

template <int KT>
__device__ __forceinline__ void update_any(Smem<KT>& s) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int cc = 0; cc < KT; ++cc) any |= s.act[cc];
        s.any = any;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- multigrid phases
__host__ __device__ constexpr int vf(int KT) { return KT >= 4 ? 4 : KT; }  // floats per thread
__host__ __device__ constexpr int vd(int KT) { return KT >= 2 ? 2 : KT; }  // doubles per thread

// first pre-smoothing sweep from x = 0: x = w D^-1 r, s = r - w (L D^-1) r
template <int KT, int V, class RT>
struct PhSmoothFirst {
    const DepthArgs& D;
    const RT* r;
    float *x, *s;
    float w;
    int c0;
    float ri[RB][V], acc[RB][V], di[RB];
    __device__ void load(int q, int i) {
        RT rv[V];
        vld<RT, V>(r + i * KT + c0, rv);
#pragma unroll
        for (int e = 0; e < V; ++e) ri[q][e] = (float)rv[e];
        ell_vec<KT, V, float>(D.col, D.LD32, D.n, D.W, i, r, c0, acc[q]);
        di[q] = __ldg(D.dinv32 + i);
    }
    __device__ void store(int q, int i) {
        float xo[V], so[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            xo[e] = w * di[q] * ri[q][e];
            so[e] = ri[q][e] - w * acc[q][e];
        }
        vst<float, V>(x + i * KT + c0, xo);
        vst<float, V>(s + i * KT + c0, so);
    }
};

// smoothing sweep: x += w D^-1 s, s' = s - w (L D^-1) s (s' skipped when last);
// optionally the partial (r, x) of the final sweep on the finest level
template <int KT, int V, class RT>
struct PhSmooth {
    const DepthArgs& D;
    const float* src;
    float *dst, *x;
    const RT* rtop;  // non-null: accumulate (r, x)
    float w;
    int c0;
    bool last;
    double rz[V];
    float si[RB][V], xi[RB][V], acc[RB][V], di[RB], ri[RB][V];
    __device__ void load(int q, int i) {
        vld<float, V>(src + i * KT + c0, si[q]);
        vld<float, V>(x + i * KT + c0, xi[q]);
        di[q] = __ldg(D.dinv32 + i);
        if (!last) ell_vec<KT, V, float>(D.col, D.LD32, D.n, D.W, i, src, c0, acc[q]);
        if (rtop) {
            RT rv[V];
            vld<RT, V>(rtop + i * KT + c0, rv);
#pragma unroll
            for (int e = 0; e < V; ++e) ri[q][e] = (float)rv[e];
        }
    }
    __device__ void store(int q, int i) {
        float xo[V];
#pragma unroll
        for (int e = 0; e < V; ++e) xo[e] = xi[q][e] + w * di[q] * si[q][e];
        vst<float, V>(x + i * KT + c0, xo);
        if (!last) {
            float so[V];
#pragma unroll
            for (int e = 0; e < V; ++e) so[e] = si[q][e] - w * acc[q][e];
            vst<float, V>(dst + i * KT + c0, so);
        }
        if (rtop) {
#pragma unroll
            for (int e = 0; e < V; ++e) rz[e] += (double)ri[q][e] * (double)xo[e];
        }
    }
};

// restriction r_c = P^T s (coarse rows)
template <int KT, int V>
struct PhRestrict {
    const DepthArgs& D;  // fine depth (holds P^T)
    const float* src;
    float* rc;
    int nc;
    int c0;
    float acc[RB][V];
    __device__ void load(int q, int ic) {
#pragma unroll
        for (int e = 0; e < V; ++e) acc[q][e] = 0.0f;
        int32_t j[WMAX];
        float a[WMAX];
#pragma unroll
        for (int w = 0; w < WMAX; ++w)
            if (w < D.rt_W) {
                j[w] = __ldg(D.rt_col + w * nc + ic);
                a[w] = __ldg(D.rt_w + w * nc + ic);
            }
#pragma unroll
        for (int w = 0; w < WMAX; ++w)
            if (w < D.rt_W) {
                float xv[V];
                vld<float, V>(src + j[w] * KT + c0, xv);
#pragma unroll
                for (int e = 0; e < V; ++e) acc[q][e] += a[w] * xv[e];
            }
        for (int w = WMAX; w < D.rt_W; ++w) {
            float xv[V];
            vld<float, V>(src + __ldg(D.rt_col + w * nc + ic) * KT + c0, xv);
            const float aw = __ldg(D.rt_w + w * nc + ic);
#pragma unroll
            for (int e = 0; e < V; ++e) acc[q][e] += aw * xv[e];
        }
    }
    __device__ void store(int q, int ic) { vst<float, V>(rc + ic * KT + c0, acc[q]); }
};

// prolongation y = P x_c, x += y
template <int KT, int V>
struct PhProlong {
    const DepthArgs& D;
    const float* xc;
    float *x, *y;
    int c0;
    float yi[RB][V], xi[RB][V];
    __device__ void load(int q, int i) {
#pragma unroll
        for (int e = 0; e < V; ++e) yi[q][e] = 0.0f;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int32_t p = __ldg(D.par + k * D.n + i);
            if (p >= 0) {
                const float wk = __ldg(D.pw + k * D.n + i);
                float xv[V];
                vld<float, V>(xc + p * KT + c0, xv);
#pragma unroll
                for (int e = 0; e < V; ++e) yi[q][e] += wk * xv[e];
            }
        }
        vld<float, V>(x + i * KT + c0, xi[q]);
    }
    __device__ void store(int q, int i) {
        float xo[V];
#pragma unroll
        for (int e = 0; e < V; ++e) xo[e] = xi[q][e] + yi[q][e];
        vst<float, V>(y + i * KT + c0, yi[q]);
        vst<float, V>(x + i * KT + c0, xo);
    }
};

// residual update after the prolongation: s -= L y
template <int KT, int V>
struct PhResUpdate {
    const DepthArgs& D;
    const float* y;
    float* s;
    int c0;
    float si[RB][V], acc[RB][V];
    __device__ void load(int q, int i) {
        vld<float, V>(s + i * KT + c0, si[q]);
        ell_vec<KT, V, float>(D.col, D.L32, D.n, D.W, i, y, c0, acc[q]);
    }
    __device__ void store(int q, int i) {
        float so[V];
#pragma unroll
        for (int e = 0; e < V; ++e) so[e] = si[q][e] - acc[q][e];
        vst<float, V>(s + i * KT + c0, so);
    }
};

// Jacobi preconditioner z = D^-1 r, partial (r, z)
template <int KT, int V, class RT>
struct PhJacobi {
    const DepthArgs& D;
    const RT* r;
    float* z;
    int c0;
    double rz[V];
    RT ri[RB][V];
    float di[RB];
    __device__ void load(int q, int i) {
        vld<RT, V>(r + i * KT + c0, ri[q]);
        di[q] = __ldg(D.dinv32 + i);
    }
    __device__ void store(int q, int i) {
        float zo[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            zo[e] = di[q] * (float)ri[q][e];
            rz[e] += (double)ri[q][e] * (double)zo[e];
        }
        vst<float, V>(z + i * KT + c0, zo);
    }
};

// Dense base solve x = A^-1 r on the deepest level: r staged transposed in shared memory.
template <int KT, class RT>
__device__ void base_solve(Ctx<KT>& c, const PcgArgs& a, int64_t n0, const RT* rin, float* xo, float* stage) {
    for (int64_t q = threadIdx.x; q < n0 * KT; q += NT) {
        int64_t j = q / KT;
        int cc = (int)(q % KT);
        stage[cc * n0 + j] = (float)ldcg(rin + q);
    }
    __syncthreads();
    int64_t rb, re;
    c.rows(n0, rb, re);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i = rb + warp; i < re; i += NWARP) {
        float acc[KT];
#pragma unroll
        for (int cc = 0; cc < KT; ++cc) acc[cc] = 0.0f;
        const float* row = a.base_inv + i * n0;
        for (int64_t j = lane; j < n0; j += 32) {
            const float aij = __ldg(row + j);
#pragma unroll
            for (int cc = 0; cc < KT; ++cc) acc[cc] += aij * stage[cc * n0 + j];
        }
        float mine = 0.0f;
#pragma unroll
        for (int cc = 0; cc < KT; ++cc) {
            float v = acc[cc];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == cc) mine = v;
        }
        if (lane < KT) stcg(xo + i * KT + lane, mine);
    }
}

// z = B r: one multigrid V-cycle (or Jacobi), z in d[0].x.  Called by every thread
// of the cluster (it contains cluster barriers).  Adds the thread's partial (r, z)
// over its depth-0 rows and columns to rz[]; ends without a barrier.
template <int KT, class RT>
__device__ void precondition(Ctx<KT>& c, const PcgArgs& a, const RT* rtop, float* stage, double (&rz)[vf(KT)]) {
    constexpr int V = vf(KT);
    const float w = a.omega;
    const int c0 = Lanes<KT, V>::c0();
    const int nu = min(a.nu, MG_MAX_NU);
    if (a.precond == 0) {
        const DepthArgs& D = a.d[0];
        PhJacobi<KT, V, RT> ph{D, rtop, c.tv(D.x, D.n), c0, {}, {}, {}};
        run_rows<KT, V>(c, D.n, ph);
#pragma unroll
        for (int e = 0; e < V; ++e) rz[e] += ph.rz[e];
        return;
    }
    int sel[MG_MAX_DEPTH];
    // ---- down: pre-smoothing and restriction
    for (int dd = 0; dd < a.nd - 1; ++dd) {
        const DepthArgs& D = a.d[dd];
        float* x = c.tv(D.x, D.n);
        float* sa = c.tv(D.sa, D.n);
        float* sb = c.tv(D.sb, D.n);
        const float* ws = a.wsm[dd];
        if (dd == 0) {
            PhSmoothFirst<KT, V, RT> ph{D, rtop, x, sa, ws[0], c0, {}, {}, {}};
            run_rows<KT, V>(c, D.n, ph);
        } else {
            PhSmoothFirst<KT, V, float> ph{D, c.tv(D.r, D.n), x, sa, ws[0], c0, {}, {}, {}};
            run_rows<KT, V>(c, D.n, ph);
        }
        c.cl.sync();
        int sl = 0;
        for (int sw = 1; sw < nu; ++sw) {
            PhSmooth<KT, V, RT> ph{D, sl ? sb : sa, sl ? sa : sb, x, nullptr, ws[sw], c0, false, {}, {}, {}, {}, {}, {}};
            run_rows<KT, V>(c, D.n, ph);
            c.cl.sync();
            sl ^= 1;
        }
        sel[dd] = sl;
        const DepthArgs& C = a.d[dd + 1];
        PhRestrict<KT, V> pr{D, sl ? sb : sa, c.tv(C.r, C.n), C.n, c0, {}};
        run_rows<KT, V>(c, C.n, pr);
        c.cl.sync();
    }
    // ---- coarsest level
    {
        const DepthArgs& B = a.d[a.nd - 1];
        float* x = c.tv(B.x, B.n);
        if (a.base_inv) {
            if (a.nd == 1) base_solve<KT, RT>(c, a, B.n, rtop, x, stage);
            else base_solve<KT, float>(c, a, B.n, c.tv(B.r, B.n), x, stage);
        } else {  // no dense inverse: one damped Jacobi sweep
            int64_t rb, re;
            c.rows(B.n, rb, re);
            for (int64_t q = rb * KT + threadIdx.x; q < re * KT; q += NT) {
                const int64_t i = q / KT;
                float ri = a.nd == 1 ? (float)ldcg(rtop + q) : ldcg(c.tv(B.r, B.n) + q);
                stcg(x + q, w * __ldg(B.dinv32 + i) * ri);
            }
        }
        if (a.nd == 1) {
            __syncthreads();
            int64_t rb, re;
            c.rows(B.n, rb, re);
            for (int64_t i = rb + Lanes<KT, V>::roff(); i < re; i += Lanes<KT, V>::RPP) {
                float xv[V];
                RT rv[V];
                vld<float, V>(x + i * KT + c0, xv);
                vld<RT, V>(rtop + i * KT + c0, rv);
#pragma unroll
                for (int e = 0; e < V; ++e) rz[e] += (double)rv[e] * (double)xv[e];
            }
            return;
        }
        c.cl.sync();
    }
    // ---- up: prolongation, residual update, post-smoothing
    for (int dd = a.nd - 2; dd >= 0; --dd) {
        const DepthArgs& D = a.d[dd];
        const DepthArgs& C = a.d[dd + 1];
        float* x = c.tv(D.x, D.n);
        float* y = c.tv(D.y, D.n);
        float* sa = c.tv(D.sa, D.n);
        float* sb = c.tv(D.sb, D.n);
        {
            PhProlong<KT, V> ph{D, c.tv(C.x, C.n), x, y, c0, {}, {}};
            run_rows<KT, V>(c, D.n, ph);
        }
        c.cl.sync();
        int sl = sel[dd];
        {
            PhResUpdate<KT, V> ph{D, y, sl ? sb : sa, c0, {}, {}};
            run_rows<KT, V>(c, D.n, ph);
        }
        c.cl.sync();
        for (int sw = 0; sw < nu; ++sw) {
            const bool last = sw == nu - 1;
            PhSmooth<KT, V, RT> ph{D, sl ? sb : sa, sl ? sa : sb, x, (last && dd == 0) ? rtop : nullptr,
                                   a.wsm[dd][nu - 1 - sw], c0, last, {}, {}, {}, {}, {}, {}};
            run_rows<KT, V>(c, D.n, ph);
            if (last && dd == 0) {
#pragma unroll
                for (int e = 0; e < V; ++e) rz[e] += ph.rz[e];
                break;
            }
            c.cl.sync();
            sl ^= 1;
        }
    }
}

// ---------------------------------------------------------------- PCG phases
// p = z + beta p, q = L z + beta q, partial (p, q)
template <int KT, int V, class T>
struct PhPcgA {
    const DepthArgs& D;
    const T* Lv;
    const float* z;
    T *p, *q;
    const double* beta;  // per column (shared memory)
    int c0;
    double pq[V];
    T lz[RB][V], pi[RB][V], qi[RB][V];
    float zi[RB][V];
    __device__ void load(int k, int i) {
        ell_vec<KT, V, T>(D.col, Lv, D.n, D.W, i, z, c0, lz[k]);
        vld<float, V>(z + i * KT + c0, zi[k]);
        vld<T, V>(p + i * KT + c0, pi[k]);
        vld<T, V>(q + i * KT + c0, qi[k]);
    }
    __device__ void store(int k, int i) {
        T po[V], qo[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const T b = (T)beta[c0 + e];
            po[e] = (T)zi[k][e] + b * pi[k][e];
            qo[e] = lz[k][e] + b * qi[k][e];
            pq[e] += (double)po[e] * (double)qo[e];
        }
        vst<T, V>(p + i * KT + c0, po);
        vst<T, V>(q + i * KT + c0, qo);
    }
};

// d += alpha p, r -= alpha q, partial (r, r)
template <int KT, int V, class T>
struct PhPcgB {
    T *d, *r;
    const T *p, *q;
    const double* alpha;
    int c0;
    double rr[V];
    T di[RB][V], ri[RB][V], pi[RB][V], qi[RB][V];
    __device__ void load(int k, int i) {
        vld<T, V>(d + i * KT + c0, di[k]);
        vld<T, V>(r + i * KT + c0, ri[k]);
        vld<T, V>(p + i * KT + c0, pi[k]);
        vld<T, V>(q + i * KT + c0, qi[k]);
    }
    __device__ void store(int k, int i) {
        T dn[V], rn[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const T al = (T)alpha[c0 + e];
            dn[e] = di[k][e] + al * pi[k][e];
            rn[e] = ri[k][e] - al * qi[k][e];
            rr[e] += (double)rn[e] * (double)rn[e];
        }
        vst<T, V>(d + i * KT + c0, dn);
        vst<T, V>(r + i * KT + c0, rn);
    }
};

// PCG on the tile for L d = r (tile-major depth-0 vectors of type T, operator Lv).
// Columns with s.act set iterate; a column stops when ||r||^2 <= tol2 * s.ref, or
// at the rounding floor ||r||^2 <= fl_stop2 * s.ss; it does not start when its
// initial residual is within fl_acc2 * s.ss (0, 0: no floor).
template <int KT, class T>
__device__ void pcg(Ctx<KT>& c, Smem<KT>& s, const PcgArgs& a, T* d, T* r, T* p, T* q, const T* Lv, double tol2,
                    double fl_stop2, double fl_acc2, float* stage) {
    constexpr int VV = std::is_same<T, double>::value ? vd(KT) : vf(KT);
    constexpr int VF = vf(KT);
    const DepthArgs& D = a.d[0];
    d = c.tv(d, D.n);
    r = c.tv(r, D.n);
    p = c.tv(p, D.n);
    q = c.tv(q, D.n);
    const float* z = c.tv(D.x, D.n);
    {
        double v[1][VV] = {};
        int64_t rb, re;
        c.rows(D.n, rb, re);
        const int c0 = Lanes<KT, VV>::c0();
        for (int64_t i = rb + Lanes<KT, VV>::roff(); i < re; i += Lanes<KT, VV>::RPP) {
            T rv[VV];
            vld<T, VV>(r + i * KT + c0, rv);
#pragma unroll
            for (int e = 0; e < VV; ++e) v[0][e] += (double)rv[e] * (double)rv[e];
        }
        cluster_sum<KT, VV, 1, double>(c, s, v);
        if (threadIdx.x < KT) {
            int cc = threadIdx.x;
            const double rr0 = s.tot[0][cc];
            if (s.act[cc] && !(rr0 - rr0 == 0.0)) {
                s.bad[cc] = 1;
                s.act[cc] = 0;
            }
            if (s.act[cc] && (rr0 <= tol2 * s.ref[cc] || rr0 <= fl_acc2 * s.ss[cc])) s.act[cc] = 0;
            s.iters[cc] = 0;
            s.beta[cc] = 0.0;
        }
        update_any(s);
    }
    for (int it = 1; it <= a.max_it && s.any; ++it) {
        // z = B r and (r, z); every thread takes part in the preconditioner's barriers
        {
            double rz[1][VF] = {};
            precondition<KT, T>(c, a, (const T*)r, stage, rz[0]);
            cluster_sum<KT, VF, 1, double>(c, s, rz);
            if (threadIdx.x < KT) {
                int cc = threadIdx.x;
                double gn = s.tot[0][cc];
                s.beta[cc] = (it == 1 || s.gam[cc] == 0.0) ? 0.0 : gn / s.gam[cc];
                s.gam[cc] = gn;
            }
            __syncthreads();
        }
        // p = z + beta p, q = L z + beta q, partial (p, q)
        {
            PhPcgA<KT, VV, T> ph{D, Lv, z, p, q, s.beta, Lanes<KT, VV>::c0(), {}, {}, {}, {}, {}};
            run_rows<KT, VV>(c, D.n, ph);
            double v[1][VV];
#pragma unroll
            for (int e = 0; e < VV; ++e) v[0][e] = ph.pq[e];
            cluster_sum<KT, VV, 1, double>(c, s, v);
            if (threadIdx.x < KT) {
                int cc = threadIdx.x;
                double pq = s.tot[0][cc];
                s.alpha[cc] = (s.act[cc] && pq != 0.0) ? s.gam[cc] / pq : 0.0;
            }
            __syncthreads();
        }
        // d += alpha p, r -= alpha q, partial (r, r)
        {
            PhPcgB<KT, VV, T> ph{d, r, p, q, s.alpha, Lanes<KT, VV>::c0(), {}, {}, {}, {}, {}};
            run_rows<KT, VV>(c, D.n, ph);
            double v[1][VV];
#pragma unroll
            for (int e = 0; e < VV; ++e) v[0][e] = ph.rr[e];
            cluster_sum<KT, VV, 1, double>(c, s, v);
            if (threadIdx.x < KT) {
                int cc = threadIdx.x;
                if (s.act[cc]) {
                    s.iters[cc] = it;
                    double rr = s.tot[0][cc];
                    if (!(rr - rr == 0.0)) s.bad[cc] = 1;
                    if (rr <= tol2 * s.ref[cc] || rr <= fl_stop2 * s.ss[cc] || !(rr - rr == 0.0)) s.act[cc] = 0;
                }
            }
            update_any(s);
        }
    }
}

// FP32+refinement: FP64 residual update of the columns with s.upd set:
// r = b - L64 (x + d) into r32, then the column's decisions (stop at the tolerance
// or the rounding floor, fail when not finite, after max_refine updates or three
// updates in a row that took less than 10 % off ||r|| above the acceptance margin), then
// x += d, d = 0 for those columns.  Called by every thread of the cluster.
template <int KT>
__device__ void reliable_update(Ctx<KT>& c, Smem<KT>& s, const PcgArgs& a) {
    const DepthArgs& D = a.d[0];
    const int lc = threadIdx.x % KT;
    const int64_t rs = NT / KT;
    int64_t rb0, re0;
    c.rows(D.n, rb0, re0);
    double* x64 = c.tv(a.x64, D.n);
    const double* b64 = c.tv(a.b64, D.n);
    float* d32 = c.tv(a.d32, D.n);
    float* r32 = c.tv(a.r32, D.n);
    const bool on = s.upd[lc] != 0;
    double v[2][1] = {{0.0}, {0.0}};
    for (int64_t i = rb0 + threadIdx.x / KT; i < re0; i += rs) {
        if (!on) continue;
        double lx = 0.0;
        float alx = 0.0f;
        for (int w = 0; w < D.W; ++w) {
            const int64_t j = __ldg(D.col + (int64_t)w * D.n + i);
            const double xj = ldcg(x64 + j * KT + lc) + (double)ldcg(d32 + j * KT + lc);
            lx += __ldg(D.L64 + (int64_t)w * D.n + i) * xj;
            alx += fabsf(__ldg(D.L32 + (int64_t)w * D.n + i)) * abs_to_float(xj);
        }
        const double bi = ldcg(b64 + i * KT + lc);
        const double ri = bi - lx;
        stcg(r32 + i * KT + lc, (float)ri);
        v[0][0] += ri * ri;
        const float si = abs_to_float(bi) + alx;
        v[1][0] += (double)(si * si);
    }
    cluster_sum<KT, 1, 2, double>(c, s, v);  // its cluster barrier also ends all reads of x and d
    if (threadIdx.x < KT) {
        const int cc = threadIdx.x;
        if (s.upd[cc] && s.outer[cc] == 1) {
            const double rr = s.tot[0][cc], sv = s.tot[1][cc];
            const bool first = s.nup[cc] == 0;
            const double fl2 = first ? a.fl_acc2 : a.fl_stop2;
            if (!(rr - rr == 0.0)) {
                s.bad[cc] = 1;
                s.outer[cc] = 2;
            } else if (rr <= a.tol * a.tol * s.bb[cc] || rr <= fl2 * sv) {
                s.outer[cc] = 0;
            } else {
                if (!first && rr > 0.81 * s.ref[cc]) s.stall[cc] += 1;
                else s.stall[cc] = 0;
                if (s.stall[cc] >= 3) s.outer[cc] = rr <= a.fl_acc2 * sv ? 0 : 2;
                else if (s.nup[cc] > a.max_refine) s.outer[cc] = 2;
            }
            // the FP32 recurrence had drifted from the true residual by more than 2x:
            // its search direction no longer fits, restart it (beta = 0)
            if (!first && rr > 4.0 * s.prev[cc]) s.gam[cc] = 0.0;
            s.nup[cc] += 1;
            s.ref[cc] = rr;
            s.lastu[cc] = s.iters[cc];
            s.act[cc] = s.outer[cc] == 1;
        }
    }
    for (int64_t i = rb0 + threadIdx.x / KT; i < re0; i += rs) {
        if (!on) continue;
        const int64_t o = i * KT + lc;
        stcg(x64 + o, ldcg(x64 + o) + (double)ldcg(d32 + o));
        stcg(d32 + o, 0.0f);
    }
    update_any(s);
}

// FP32 PCG with reliable updates (FP32+refinement form): the FP32 recurrence runs
// on across FP64 residual replacements; a column whose FP32 residual has fallen by
// inner_tol since its last FP64 residual, or below the tolerance, is updated.
template <int KT>
__device__ void pcg_ru(Ctx<KT>& c, Smem<KT>& s, const PcgArgs& a, float* stage) {
    constexpr int VF = vf(KT);
    const DepthArgs& D = a.d[0];
    float* d = c.tv(a.d32, D.n);
    float* r = c.tv(a.r32, D.n);
    float* p = c.tv(a.p32, D.n);
    float* q = c.tv(a.q32, D.n);
    const float* z = c.tv(D.x, D.n);
    if (threadIdx.x < KT) {
        s.upd[threadIdx.x] = s.outer[threadIdx.x] == 1;
        s.beta[threadIdx.x] = 0.0;
    }
    __syncthreads();
    reliable_update<KT>(c, s, a);
    for (int it = 1; it <= a.max_it && s.any; ++it) {
        {
            double rz[1][VF] = {};
            precondition<KT, float>(c, a, (const float*)r, stage, rz[0]);
            cluster_sum<KT, VF, 1, double>(c, s, rz);
            if (threadIdx.x < KT) {
                int cc = threadIdx.x;
                double gn = s.tot[0][cc];
                s.beta[cc] = (it == 1 || s.gam[cc] == 0.0) ? 0.0 : gn / s.gam[cc];
                s.gam[cc] = gn;
            }
            __syncthreads();
        }
        {
            PhPcgA<KT, VF, float> ph{D, D.L32, z, p, q, s.beta, Lanes<KT, VF>::c0(), {}, {}, {}, {}, {}};
            run_rows<KT, VF>(c, D.n, ph);
            double v[1][VF];
#pragma unroll
            for (int e = 0; e < VF; ++e) v[0][e] = ph.pq[e];
            cluster_sum<KT, VF, 1, double>(c, s, v);
            if (threadIdx.x < KT) {
                int cc = threadIdx.x;
                double pq = s.tot[0][cc];
                s.alpha[cc] = (s.act[cc] && pq != 0.0) ? s.gam[cc] / pq : 0.0;
            }
            __syncthreads();
        }
        {
            PhPcgB<KT, VF, float> ph{d, r, p, q, s.alpha, Lanes<KT, VF>::c0(), {}, {}, {}, {}, {}};
            run_rows<KT, VF>(c, D.n, ph);
            double v[1][VF];
#pragma unroll
            for (int e = 0; e < VF; ++e) v[0][e] = ph.rr[e];
            cluster_sum<KT, VF, 1, double>(c, s, v);
            if (threadIdx.x < KT) {
                int cc = threadIdx.x;
                int u = 0;
                if (s.act[cc]) {
                    s.iters[cc] = it;
                    const double rr = s.tot[0][cc];
                    if (!(rr - rr == 0.0)) {
                        s.bad[cc] = 1;
                        s.act[cc] = 0;
                        s.outer[cc] = 2;
                    } else {
                        u = rr <= a.inner_tol * a.inner_tol * s.ref[cc] || rr <= a.tol * a.tol * s.bb[cc] ||
                            s.iters[cc] - s.lastu[cc] >= kMaxInner;
                        if (u) s.prev[cc] = rr;  // the FP32 residual the FP64 one is compared with
                    }
                }
                s.upd[cc] = u;
            }
            __syncthreads();
            int anyu = 0;
            for (int cc = 0; cc < KT; ++cc) anyu |= s.upd[cc];
            if (anyu) reliable_update<KT>(c, s, a);
            else update_any(s);
        }
    }
}

// ---------------------------------------------------------------- the kernel
template <int KT, int MODE>
__global__ void __launch_bounds__(NT, MG_MINB) k_phi_batch(PcgArgs a) {
    __shared__ Smem<KT> s;
    extern __shared__ float stage[];
    Ctx<KT> c;
    const DepthArgs& D = a.d[0];
    const int c0 = c.tile * KT;
    const int kc = min(KT, a.k - c0);
    // scalar mapping (one column per thread) for the once-per-launch phases
    const int lc = threadIdx.x % KT;
    const int64_t rs = NT / KT;
    const bool valid = lc < kc;
    const int64_t cio = c0 + lc;
    int64_t rb0, re0;
    c.rows(D.n, rb0, re0);

    double sg[3] = {0.0, 0.0, 0.0};
    if (valid) {
        const int64_t t = a.t0 + cio * a.tstride;
        for (int q = 0; q < 3; ++q) sg[q] = a.wave[3 * t + q];
    }
    if (threadIdx.x < KT) {
        s.act[threadIdx.x] = threadIdx.x < kc;
        s.outer[threadIdx.x] = threadIdx.x < kc;
        s.iters[threadIdx.x] = 0;
        s.bad[threadIdx.x] = 0;
        s.gam[threadIdx.x] = 0.0;
    }
    __syncthreads();

    double* x64 = c.tv(a.x64, D.n);
    // ---- b = (1/dt) M x_prev + J0 sum_s b_s F_s, x0 = guess - g; FP64 form: r = b - L x0.
    // Every column of the tile is initialised (columns past k with zeros).
    {
        double v[2][1] = {{0.0}, {0.0}};  // ||b||^2 and, FP64 form, S^2 of the rounding floor
        double* r64 = a.mode == 0 ? c.tv(a.r64, D.n) : nullptr;
        double* b64 = a.mode == 1 ? c.tv(a.b64, D.n) : nullptr;
        float* z = c.tv(D.x, D.n);
        for (int64_t i = rb0 + threadIdx.x / KT; i < re0; i += rs) {
            double bi = 0.0, lx = 0.0, xi = 0.0;
            float alx = 0.0f;  // sum |L_ij| |x_j| of the rounding floor (an estimate: FP32)
            if (valid) {
                double mb = 0.0;
                for (int wq = 0; wq < D.W; ++wq) {
                    const int64_t j = __ldg(D.col + (int64_t)wq * D.n + i);
                    mb += __ldg(D.M64 + (int64_t)wq * D.n + i) * a.xprev[j * a.ld_prev + cio];
                    if (a.guess) {
                        double xj = a.guess[j * a.ld_guess + cio];
                        if (a.g) xj -= a.g[j * a.ld_g + cio];
                        lx += __ldg(D.L64 + (int64_t)wq * D.n + i) * xj;
                        alx += fabsf(__ldg(D.L32 + (int64_t)wq * D.n + i)) * abs_to_float(xj);
                    }
                }
                bi = mb * a.inv_dt + a.J0 * (sg[0] * a.F[i] + sg[1] * a.F[D.n + i] + sg[2] * a.F[2 * D.n + i]);
                if (a.guess) {
                    xi = a.guess[i * a.ld_guess + cio];
                    if (a.g) xi -= a.g[i * a.ld_g + cio];
                }
            }
            const int64_t o = i * KT + lc;
            stcg(x64 + o, xi);
            stcg(z + o, 0.0f);
            if (a.mode == 0) {
                stcg(r64 + o, bi - lx);
                stcg(c.tv(a.p64, D.n) + o, 0.0);
                stcg(c.tv(a.q64, D.n) + o, 0.0);
            } else {
                stcg(b64 + o, bi);
            }
            v[0][0] += bi * bi;
            const float si = abs_to_float(bi) + alx;
            v[1][0] += (double)(si * si);
        }
        cluster_sum<KT, 1, 2, double>(c, s, v);
        if (threadIdx.x < KT) {
            s.bb[threadIdx.x] = s.tot[0][threadIdx.x];
            s.ss[threadIdx.x] = s.tot[1][threadIdx.x];
        }
        __syncthreads();
    }

    if constexpr (MODE == 0) {
        if (threadIdx.x < KT) s.ref[threadIdx.x] = s.bb[threadIdx.x];
        __syncthreads();
        pcg<KT, double>(c, s, a, a.x64, a.r64, a.p64, a.q64, D.L64, a.tol * a.tol, a.fl_stop2, a.fl_acc2, stage);
        if (threadIdx.x < KT) s.outer[threadIdx.x] = s.act[threadIdx.x];
        __syncthreads();
    } else {
        // d = p = q = 0 (the initial FP64 residual comes from the first update)
        for (int64_t i = rb0 + threadIdx.x / KT; i < re0; i += rs) {
            const int64_t o = i * KT + lc;
            stcg(c.tv(a.d32, D.n) + o, 0.0f);
            stcg(c.tv(a.p32, D.n) + o, 0.0f);
            stcg(c.tv(a.q32, D.n) + o, 0.0f);
        }
        if (threadIdx.x < KT) {
            s.nup[threadIdx.x] = 0;
            s.stall[threadIdx.x] = 0;
            s.lastu[threadIdx.x] = 0;
        }
        c.cl.sync();
        pcg_ru<KT>(c, s, a, stage);
    }

    // ---- x_out = x (+ d not yet folded in) + g; per-column status
    c.cl.sync();
    if (valid) {
        for (int64_t i = rb0 + threadIdx.x / KT; i < re0; i += rs) {
            double xi = ldcg(x64 + i * KT + lc);
            if (a.mode == 1) xi += (double)ldcg(c.tv(a.d32, D.n) + i * KT + lc);
            if (a.g) xi += a.g[i * a.ld_g + cio];
            a.xout[i * a.ld_out + cio] = xi;
        }
    }
    if (c.rank == 0 && threadIdx.x < kc) {
        int cc = threadIdx.x;
        if (s.bad[cc]) atomicMin(a.worst, (int)MG_ENONFINITE);
        else if (s.outer[cc]) atomicMin(a.worst, (int)MG_ECG_MAXIT);
        atomicAdd(a.iter_sum, (unsigned long long)s.iters[cc]);
    }
}

// Largest cluster size <= want (16 or 8) that the device can schedule for this kernel.
template <int KT, int MODE>
int usable_cluster(int want, size_t stage_bytes) {
    static int cached[17] = {};
    if (want <= 8) return want;
    if (cached[want]) return cached[want];
    MG_CUDA(cudaFuncSetAttribute(k_phi_batch<KT, MODE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    MG_CUDA(cudaFuncSetAttribute(k_phi_batch<KT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(stage_bytes, 64 * 1024)));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(want);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = std::max<size_t>(stage_bytes, 64 * 1024);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = want;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, k_phi_batch<KT, MODE>, &cfg);
    cudaGetLastError();
    cached[want] = (e == cudaSuccess && n > 0) ? want : 8;
    return cached[want];
}

template <int KT, int MODE>
void launch_mode(const PcgArgs& a, int csize, size_t stage_bytes, cudaStream_t stream) {
    const int ntile = (a.k + KT - 1) / KT;
    csize = usable_cluster<KT, MODE>(csize, stage_bytes);
    MG_CUDA(cudaFuncSetAttribute(k_phi_batch<KT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)stage_bytes));
    if (csize > 8) MG_CUDA(cudaFuncSetAttribute(k_phi_batch<KT, MODE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntile * csize));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = stage_bytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MG_CUDA(cudaLaunchKernelEx(&cfg, k_phi_batch<KT, MODE>, a));
}

template <int KT>
void launch(const PcgArgs& a, int csize, size_t stage_bytes, cudaStream_t stream) {
    if (a.mode == 0) launch_mode<KT, 0>(a, csize, stage_bytes, stream);
    else launch_mode<KT, 1>(a, csize, stage_bytes, stream);
}

}  // namespace

static int choose_tile(int k, int want) {
    if (want == 1 || want == 8 || want == 16 || want == 32) return want;
    if (k <= 1) return 1;
    if (k <= 8) return 8;
    return 16;
}

void phi_batch(mg_ctx* c, const StepOp& op, const PhiIO& io, const mg_solver_opts& so, SolveCounters* counters) {
    if (io.k <= 0) return;
    // the kernels add their PCG iterations and statuses to the context counters;
    // a caller that did not reset them (the autotuner) may come first
    if (!c->counters.p) {
        c->counters.ensure(16);
        MG_CUDA(cudaMemsetAsync(c->counters.p, 0, 16, c->stream));
    }
    if (so.max_cg < 1 || so.max_refine < 0 || (so.precision != MG_FP64 && so.precision != MG_FP32_REFINE) ||
        (so.precond != MG_PRECOND_JACOBI && so.precond != MG_PRECOND_MULTIGRID))
        mg_fail(MG_EINVAL, "bad solver options");
    if (mesh_is_nonlinear(c, op.mesh)) {
        phi_batch_newton(c, op, io, so, counters);
        return;
    }
    if (so.path == MG_PATH_AUTO && so.tile == 0 && so.cluster == 0 && so.rows_per_block == 0 &&
        so.coarse_rows_per_block == 0 && so.base_tiles == 0 && so.halo_fusion == 0 && so.base_cores == 0) {
        // a launch shape mg_autotune recorded for this mesh and tile count
        auto it = c->tuned.find({op.mesh, tune_bucket(io.k)});
        if (it != c->tuned.end()) {
            mg_solver_opts t = so;
            t.path = it->second.path;
            t.tile = it->second.tile;
            t.cluster = it->second.cluster;
            t.rows_per_block = it->second.rbs0;
            t.coarse_rows_per_block = it->second.rbs1;
            t.base_tiles = it->second.base_tiles;
            t.halo_fusion = it->second.hf;
            t.base_cores = it->second.bc;
            phi_batch(c, op, io, t, counters);
            return;
        }
    }
    if (so.path == MG_PATH_GRAPH || (so.path == MG_PATH_AUTO && io.k >= MG_GRAPH_MIN_COLUMNS)) {
        phi_batch_graph(c, op, io, so, counters);
        return;
    }
    const MeshLevel& m0 = c->meshes[op.mesh];
    const int KT = choose_tile(io.k, so.tile);
    const int ntile = (io.k + KT - 1) / KT;
    // one tile: the largest cluster (latency-bound); several: 8 CTAs so more clusters fit
    int csize = so.cluster > 0 ? so.cluster : (ntile == 1 ? 16 : 8);
    csize = std::max(1, std::min(16, csize));
    PcgArgs a = {};
    a.precond = so.precond;
    a.nu = smooth_sweeps(so);
    a.omega = so.omega > 0.0 ? (float)so.omega : 0.7f;
    a.nd = a.precond == 1 ? (int)op.mg.size() : 1;
    for (int d = 0; d < a.nd; ++d) smoother_weights(op.mg[d]->lam, so, a.nu, a.wsm[d]);
    a.base_inv = (a.precond == 1 && op.base_inv.p) ? op.base_inv.as<float>() : nullptr;
    // work vectors: each is ntile * n_d * KT elements
    int wsi = 0;
    auto grab = [&](size_t bytes) -> void* {
        if (wsi >= (int)(sizeof(c->ws) / sizeof(c->ws[0]))) mg_fail(MG_EINVAL, "too many work vectors");
        c->ws[wsi].ensure(bytes);
        return c->ws[wsi++].p;
    };
    const size_t e0 = (size_t)ntile * m0.n * KT;
    if (so.precision == MG_FP64) {
        a.x64 = (double*)grab(e0 * 8);
        a.r64 = (double*)grab(e0 * 8);
        a.p64 = (double*)grab(e0 * 8);
        a.q64 = (double*)grab(e0 * 8);
    } else {
        a.x64 = (double*)grab(e0 * 8);
        a.b64 = (double*)grab(e0 * 8);
        a.d32 = (float*)grab(e0 * 4);
        a.r32 = (float*)grab(e0 * 4);
        a.p32 = (float*)grab(e0 * 4);
        a.q32 = (float*)grab(e0 * 4);
    }
    for (int d = 0; d < a.nd; ++d) {
        const MgDepth& md = *op.mg[d];
        const MeshLevel& mm = c->meshes[md.mesh];
        DepthArgs& da = a.d[d];
        da.n = md.n;
        da.W = md.W;
        da.col = mm.ell_col.as<int32_t>();
        da.L64 = md.L64.as<double>();
        da.M64 = md.M64.as<double>();
        da.L32 = md.L32.as<float>();
        da.LD32 = md.LD32.as<float>();
        da.dinv64 = md.dinv64.as<double>();
        da.dinv32 = md.dinv32.as<float>();
        if (d + 1 < a.nd) {
            da.par = mm.par.as<int32_t>();
            da.pw = mm.pw.as<float>();
            da.rt_W = mm.rt_W;
            da.rt_col = mm.rt_col.as<int32_t>();
            da.rt_w = mm.rt_w.as<float>();
        }
        const size_t ed = (size_t)ntile * md.n * KT;
        da.x = (float*)grab(ed * 4);
        if (a.precond == 1 && d + 1 < a.nd) {
            da.sa = (float*)grab(ed * 4);
            da.sb = (float*)grab(ed * 4);
            da.y = (float*)grab(ed * 4);
        }
        if (d > 0) da.r = (float*)grab(ed * 4);
    }
    size_t stage_bytes = a.base_inv ? (size_t)a.d[a.nd - 1].n * KT * sizeof(float) : 0;
    if (stage_bytes > 200 * 1024) mg_fail(MG_EINVAL, "base mesh too large for the dense coarse solve of this tile");
    a.inv_dt = 1.0 / op.dt;
    a.F = m0.F.as<double>();
    a.J0 = c->pwm.J0;
    a.wave = io.wave;
    a.t0 = io.t0;
    a.tstride = io.tstride;
    a.xprev = io.xprev;
    a.ld_prev = io.ld_prev;
    a.g = io.g;
    a.ld_g = io.ld_g;
    a.guess = io.guess;
    a.ld_guess = io.ld_guess;
    a.xout = io.xout;
    a.ld_out = io.ld_out;
    a.k = io.k;
    a.tol = so.precision == MG_FP64 ? so.cg_tol : so.refine_tol;
    a.inner_tol = so.inner_tol;
    a.fl_stop2 = residual_floor(a.d[0].W) * residual_floor(a.d[0].W);
    a.fl_acc2 = a.fl_stop2 * kFloorAccept * kFloorAccept;
    a.max_it = so.max_cg;
    a.max_refine = so.max_refine;
    a.mode = so.precision == MG_FP64 ? 0 : 1;
    a.iter_sum = (unsigned long long*)c->counters.p;
    a.worst = (int*)((char*)c->counters.p + 8);
    switch (KT) {
        case 1: launch<1>(a, csize, stage_bytes, c->stream); break;
        case 8: launch<8>(a, csize, stage_bytes, c->stream); break;
        case 16: launch<16>(a, csize, stage_bytes, c->stream); break;
        default: launch<32>(a, csize, stage_bytes, c->stream); break;
    }
    if (counters) {
        counters->step_solves += io.k;
        counters->batched_steps += 1;
        counters->launches += 1;
    }
}

// ---------------------------------------------------------------- mg_step_static
// A batched step whose work vectors live in one fixed, file-scope device array
// instead of buffers the context allocates, for callers that must not allocate
// device memory (see include/mgrit_em.h).  The array is per device and shared by
// every call: calls whose kernels overlap on the GPU (other streams, other host
// threads) race on it.
#define MG_STATIC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_step_scratch[MG_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_step_scratch on the current device (looked up once per device).
void* static_scratch(int device) {
    if (device < 0 || device >= kMaxDevices) mg_fail(MG_EINVAL, "device id out of range for the static scratch");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_step_scratch);
        if (e != cudaSuccess || !p)
            mg_fail(MG_ECUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
        g_scratch_addr[device] = p;
    }
    return g_scratch_addr[device];
}

}  // namespace

extern mg_status mg_guarded_call(mg_ctx* c, void (*fn)(void*), void* arg);

namespace {
struct StaticStepCall {
    mg_ctx* c;
    int level;
    int64_t N;
    double T;
    int64_t dt_mult;
    int k;
    int64_t i0, istride;
    const double* x_in;
    int64_t ld_in;
    double* x_out;
    int64_t ld_out;
    int guess;
    const mg_solver_opts* opts;
    mg_stats* stats;
    mg_status result;
};

void static_step(void* arg) {
    StaticStepCall& q = *(StaticStepCall*)arg;
    mg_ctx* c = q.c;
    q.result = MG_OK;
    mg_solver_opts so;
    if (q.opts) so = *q.opts;
    else mg_solver_defaults(&so);
    if (q.level < 0 || q.level >= (int)c->meshes.size() || q.N <= 0 || !(q.T > 0.0) || q.dt_mult <= 0 || q.k <= 0 ||
        !q.x_in || !q.x_out || q.ld_in < q.k || q.ld_out < q.k || q.i0 < 0 || q.i0 > q.N || q.istride < 0 ||
        q.i0 + (int64_t)(q.k - 1) * q.istride > q.N)
        mg_fail(MG_EINVAL, "mg_step_static: bad arguments");
    check_solver_opts(so);
    const double dt = (double)q.dt_mult * q.T / (double)q.N;
    const StepOp* op = ctx_find_step_op(c, q.level, dt);
    const double* wave = ctx_find_wave_table(c, q.N, q.T, 0);
    if (!op || !wave)
        mg_fail(MG_ESTATE, "mg_step_static: the step operator or PWM table for this level, N, T and dt does not exist "
                           "yet; one regular mg_step call with the same arguments builds both");
    if (mesh_is_nonlinear(c, op->mesh))
        mg_fail(MG_EINVAL, "mg_step_static: nonlinear (Newton) steps need per-column Jacobian storage; use mg_step");
    const MeshLevel& m0 = c->meshes[op->mesh];
    const int KT = choose_tile(q.k, so.tile);
    const int csize = std::max(1, std::min(16, so.cluster > 0 ? so.cluster : 8));
    const int ntile = (q.k + KT - 1) / KT;
    PcgArgs a = {};
    a.precond = so.precond;
    a.nu = smooth_sweeps(so);
    a.omega = so.omega > 0.0 ? (float)so.omega : 0.7f;
    a.nd = a.precond == 1 ? (int)op->mg.size() : 1;
    for (int d = 0; d < a.nd; ++d) smoother_weights(op->mg[d]->lam, so, a.nu, a.wsm[d]);
    a.base_inv = (a.precond == 1 && op->base_inv.p) ? op->base_inv.as<float>() : nullptr;
    // carve the work vectors out of the static array (256-byte aligned pieces)
    const size_t e0 = (size_t)ntile * m0.n * KT;
    std::vector<size_t> need;
    if (so.precision == MG_FP64) need = {e0 * 8, e0 * 8, e0 * 8, e0 * 8};
    else need = {e0 * 8, e0 * 8, e0 * 4, e0 * 4, e0 * 4, e0 * 4};
    for (int d = 0; d < a.nd; ++d) {
        const size_t ed = (size_t)ntile * op->mg[d]->n * KT * 4;
        need.push_back(ed);
        if (a.precond == 1 && d + 1 < a.nd) {
            need.push_back(ed);
            need.push_back(ed);
            need.push_back(ed);
        }
        if (d > 0) need.push_back(ed);
    }
    size_t total = 256;  // counters
    for (size_t b : need) total += (b + 255) / 256 * 256;
    if (total > MG_STATIC_SCRATCH_BYTES)
        mg_fail(MG_EINVAL, "mg_step_static: this step needs " + std::to_string(total) +
                               " bytes of scratch; the static array holds " +
                               std::to_string((size_t)MG_STATIC_SCRATCH_BYTES) + " (use fewer columns or mg_step)");
    char* base = (char*)static_scratch(c->device);
    char* p = base + 256;
    size_t qi = 0;
    auto take = [&]() -> void* {
        void* r = p;
        p += (need[qi++] + 255) / 256 * 256;
        return r;
    };
    if (so.precision == MG_FP64) {
        a.x64 = (double*)take();
        a.r64 = (double*)take();
        a.p64 = (double*)take();
        a.q64 = (double*)take();
    } else {
        a.x64 = (double*)take();
        a.b64 = (double*)take();
        a.d32 = (float*)take();
        a.r32 = (float*)take();
        a.p32 = (float*)take();
        a.q32 = (float*)take();
    }
    for (int d = 0; d < a.nd; ++d) {
        const MgDepth& md = *op->mg[d];
        const MeshLevel& mm = c->meshes[md.mesh];
        DepthArgs& da = a.d[d];
        da.n = (int)md.n;
        da.W = md.W;
        da.col = mm.ell_col.as<int32_t>();
        da.L64 = md.L64.as<double>();
        da.M64 = md.M64.as<double>();
        da.L32 = md.L32.as<float>();
        da.LD32 = md.LD32.as<float>();
        da.dinv64 = md.dinv64.as<double>();
        da.dinv32 = md.dinv32.as<float>();
        if (d + 1 < a.nd) {
            da.par = mm.par.as<int32_t>();
            da.pw = mm.pw.as<float>();
            da.rt_W = mm.rt_W;
            da.rt_col = mm.rt_col.as<int32_t>();
            da.rt_w = mm.rt_w.as<float>();
        }
        da.x = (float*)take();
        if (a.precond == 1 && d + 1 < a.nd) {
            da.sa = (float*)take();
            da.sb = (float*)take();
            da.y = (float*)take();
        }
        if (d > 0) da.r = (float*)take();
    }
    const size_t stage_bytes = a.base_inv ? (size_t)a.d[a.nd - 1].n * KT * sizeof(float) : 0;
    if (stage_bytes > 200 * 1024) mg_fail(MG_EINVAL, "mg_step_static: base mesh too large for the dense coarse solve");
    a.inv_dt = 1.0 / op->dt;
    a.F = m0.F.as<double>();
    a.J0 = c->pwm.J0;
    a.wave = wave;
    a.t0 = q.i0;
    a.tstride = q.istride;
    a.xprev = q.x_in;
    a.ld_prev = q.ld_in;
    a.g = nullptr;
    a.ld_g = 0;
    a.guess = q.guess ? q.x_out : nullptr;
    a.ld_guess = q.ld_out;
    a.xout = q.x_out;
    a.ld_out = q.ld_out;
    a.k = q.k;
    a.tol = so.precision == MG_FP64 ? so.cg_tol : so.refine_tol;
    a.inner_tol = so.inner_tol;
    a.fl_stop2 = residual_floor(a.d[0].W) * residual_floor(a.d[0].W);
    a.fl_acc2 = a.fl_stop2 * kFloorAccept * kFloorAccept;
    a.max_it = so.max_cg;
    a.max_refine = so.max_refine;
    a.mode = so.precision == MG_FP64 ? 0 : 1;
    a.iter_sum = (unsigned long long*)base;
    a.worst = (int*)(base + 8);
    // the counters are the only scratch a step reads before writing it
    MG_CUDA(cudaMemsetAsync(base, 0, 16, c->stream));
    switch (KT) {
        case 1: launch<1>(a, csize, stage_bytes, c->stream); break;
        case 8: launch<8>(a, csize, stage_bytes, c->stream); break;
        case 16: launch<16>(a, csize, stage_bytes, c->stream); break;
        default: launch<32>(a, csize, stage_bytes, c->stream); break;
    }
    if (q.stats) {
        unsigned char h[16];
        MG_CUDA(cudaMemcpyAsync(h, base, 16, cudaMemcpyDeviceToHost, c->stream));
        MG_CUDA(cudaStreamSynchronize(c->stream));
        unsigned long long it;
        int worst;
        memcpy(&it, h, 8);
        memcpy(&worst, h + 8, 4);
        memset(q.stats, 0, sizeof(*q.stats));
        q.stats->cg_iters = (int64_t)it;
        q.stats->worst_status = worst;
        q.stats->step_solves = q.k;
        q.stats->batched_steps = 1;
        q.stats->launches = 1;
        if (worst != 0) q.result = (mg_status)worst;
    }
}
}  // namespace

extern "C" mg_status mg_step_static(mg_ctx* c, int level, int64_t N, double T, int64_t dt_mult, int k, int64_t i0,
                                    int64_t istride, const double* x_in, int64_t ld_in, double* x_out,
                                    int64_t ld_out, int guess, const mg_solver_opts* opts, mg_stats* stats) {
    StaticStepCall q{c, level, N, T, dt_mult, k, i0, istride, x_in, ld_in, x_out, ld_out, guess, opts, stats, MG_OK};
    mg_status st = mg_guarded_call(c, static_step, &q);
    return st != MG_OK ? st : q.result;
}
