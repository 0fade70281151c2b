// Batched backward-Euler steps for meshes with nonlinear (Brauer-law) materials.
//
// Sec. 5: on elements of a nonlinear region the reluctivity depends on the flux
// density, nu(|B|^2) = k1 exp(k2 |B|^2) + k3 with |B|^2 = |grad a|^2, so one step
// of Eq. discrete_system is the nonlinear system
//     F(a) = (M/dt)(a - a_prev) + K(a) a - f(t) = 0,
// solved per column by damped Newton started at a_prev (with a caller's guess, at
// whichever of the guess and a_prev has the smaller residual):
//     J(a) delta = -F(a),  J(a) = M/dt + sum_T |T| G (nu I + 2 nu' g g^T) G^T,
// where g = G^T a_T is the element gradient and nu' = d nu / d|B|^2.  The full
// correction is taken, and the step ends, once ||delta|| <= newton_tol ||a + delta||;
// otherwise the step length starts at 1 and is halved while ||F|| would grow.
//
// GPU layout: all per-column data is tile-major with 16 columns per tile, like the
// graph path of the linear step.  Each Newton iteration
//   1. evaluates nu and the element tensors N_T = |T| (nu I + 2 nu' g g^T) for every
//      nonlinear element and column,
//   2. assembles the column's Jacobian on the shared ELL pattern (constant part
//      M/dt + K of the linear elements, plus the N_T contributions),
//   3. forms the multigrid hierarchy of the column: coarse operators are Galerkin
//      products P^T J P on the nested meshes (for nested P1 elements this equals
//      re-assembling with area-averaged tensors N_T), and a banded Cholesky factor
//      of the base mesh operator,
//   4. solves J delta = -F with the graph path's PCG, which takes per-column
//      operators at every depth,
//   5. runs the step-length search: trial point, element residual, one decision
//      kernel per round; the host reads two flags per round.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"
#define MG_L1 1
#include "vec.cuh"

// Static data of one mesh for Newton steps.
struct NlMesh {
    int mesh = -1;
    int64_t ne = 0;                    // nonlinear elements
    DBuf eid;                          // int32 ne: element id on the mesh
    DBuf edof;                         // int32 3 ne: dofs of the vertices (-1 on Dirichlet nodes)
    DBuf inc_ptr, inc_src;             // dof -> 3 * (nonlinear element) + vertex
    DBuf jc_ptr, jc_e, jc_w;           // ELL entry -> nonlinear element, tensor weights (3 doubles)
    DBuf Kc;                           // ELL stiffness of the linear-law elements
    DBuf gal_ptr, gal_src, gal_w;      // parent mesh ELL entry -> (ELL entry here, weight)
    int band_u = -1, band_stride = 0;  // bandwidth of the interior operator
};

void nl_mesh_delete(NlMesh* p) { delete p; }

namespace {

using namespace mgv;

constexpr int G = MG_TILE;
constexpr int NTB = 256;
constexpr int RBS = 256;

inline unsigned nblk(int64_t n, int t = NTB) { return (unsigned)((n + t - 1) / t); }

// per-block, per-column partial sums of a 1-column-per-thread kernel
__device__ __forceinline__ void partial_col(double v, double* part) {
    __shared__ double red[NTB / 32][G];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    if (lane < G) red[warp][lane] = v;
    __syncthreads();
    if (threadIdx.x < G) {
        double s = 0.0;
        for (int w = 0; w < NTB / 32; ++w) s += red[w][threadIdx.x];
        part[(size_t)blockIdx.x * G + threadIdx.x] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double col_sum(const double* part, int nrb, int gc) {
    const int t = gc / G, l = gc % G;
    double s = 0.0;
    for (int rb = 0; rb < nrb; ++rb) s += part[((size_t)t * nrb + rb) * G + l];
    return s;
}

// Newton state of a column
enum : int { ST_IDLE = 0, ST_SOLVE = 1, ST_TRIAL = 2, ST_FAILED = 3 };

struct Cols {
    int* state;
    int* accept;
    int* halv;
    int* its;
    int* first;
    double* step;
    double* nr2;  // ||F||^2 at the accepted iterate
    int* flags;   // [0] any trial pending, [1] any column needs a Newton direction, [2] sum of iterations
};

struct Step {
    int n, W, nrb, k;
    const int32_t* col;  // ELL pattern (W x n, column-major)
    const double* M64;   // ELL mass values
    const double* Kc;    // ELL stiffness of linear elements
    const double* F;     // 3 x n phase loads
    double inv_dt, J0;
    const double* wave;
    int64_t t0, tstride;
};

// a = start iterate, a_prev = x_prev (tile-major)
__global__ void __launch_bounds__(NTB) kn_init(Step S, const double* __restrict__ xprev, int64_t ld_prev,
                                               const double* __restrict__ guess, int64_t ld_guess,
                                               const double* __restrict__ g, int64_t ld_g, double* a, double* aprev) {
    const int t = blockIdx.x / S.nrb, rb = blockIdx.x % S.nrb;
    const int lc = threadIdx.x % G, gc = t * G + lc;
    const bool valid = gc < S.k;
    const int i1 = min(S.n, (rb + 1) * RBS);
    for (int i = rb * RBS + threadIdx.x / G; i < i1; i += NTB / G) {
        double xp = 0.0, x0 = 0.0;
        if (valid) {
            xp = xprev[(int64_t)i * ld_prev + gc];
            x0 = xp;
            if (guess) {
                x0 = guess[(int64_t)i * ld_guess + gc];
                if (g) x0 -= g[(int64_t)i * ld_g + gc];
            }
        }
        const size_t o = ((size_t)t * S.n + i) * G + lc;
        aprev[o] = xp;
        a[o] = x0;
    }
}

__global__ void kn_state_init(Cols C, int k, int kpad) {
    for (int c = threadIdx.x; c < kpad; c += blockDim.x) {
        C.state[c] = c < k ? ST_SOLVE : ST_IDLE;
        C.accept[c] = 0;
        C.halv[c] = 0;
        C.its[c] = 0;
        C.first[c] = 0;
        C.step[c] = 1.0;
        C.nr2[c] = 0.0;
    }
}

struct Elems {
    int64_t ne;
    const int32_t* eid;
    const int32_t* edof;
    const double* grad;  // 6 per element of the mesh
    const double* area;
    const double* kk;    // k1, k2, k3 per element of the mesh
    int n;               // dofs of the mesh
};

// MODE 0: y_v = nu |T| G_v . g (the element's part of K(a) a) for the columns in
// state `want`; MODE 1: N = |T| (nu I + 2 nu' g g^T) for the columns in state SOLVE
// (the others need no new Jacobian; their Jacobian buffers keep older, finite values).
// Output ((t * 3 + v) * ne + e) * G + lane.
template <int MODE>
__global__ void __launch_bounds__(NTB) kn_elem(Elems E, const double* __restrict__ a, const int* __restrict__ state,
                                               int want, double* __restrict__ out) {
    const int t = blockIdx.y;
    const int lc = threadIdx.x % G, gc = t * G + lc;
    const int64_t e = (int64_t)blockIdx.x * (NTB / G) + threadIdx.x / G;
    if (e >= E.ne) return;
    if (state[gc] != (MODE == 0 ? want : (int)ST_SOLVE)) return;
    const int id = __ldg(E.eid + e);
    const double* gr = E.grad + 6 * (int64_t)id;
    double gx = 0.0, gy = 0.0, Gx[3], Gy[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        Gx[v] = __ldg(gr + 2 * v);
        Gy[v] = __ldg(gr + 2 * v + 1);
        const int d = __ldg(E.edof + 3 * e + v);
        const double av = d >= 0 ? a[((size_t)t * E.n + d) * G + lc] : 0.0;
        gx += av * Gx[v];
        gy += av * Gy[v];
    }
    const double b2 = gx * gx + gy * gy;
    const double k1 = __ldg(E.kk + 3 * id), k2 = __ldg(E.kk + 3 * id + 1), k3 = __ldg(E.kk + 3 * id + 2);
    const double ex = k1 == 0.0 ? 0.0 : exp(k2 * b2);  // k1 = 0: the law is nu = k3 exactly
    const double nu = k1 == 0.0 ? k3 : k1 * ex + k3;
    const double A = __ldg(E.area + id);
    const size_t base = ((size_t)t * 3 * E.ne + e) * G + lc;
    const size_t vs = (size_t)E.ne * G;
    if (MODE == 0) {
#pragma unroll
        for (int v = 0; v < 3; ++v) out[base + v * vs] = nu * A * (Gx[v] * gx + Gy[v] * gy);
    } else {
        const double dnu = k1 == 0.0 ? 0.0 : k1 * k2 * ex;
        out[base] = A * (nu + 2.0 * dnu * gx * gx);
        out[base + vs] = A * (2.0 * dnu * gx * gy);
        out[base + 2 * vs] = A * (nu + 2.0 * dnu * gy * gy);
    }
}

// R = (M/dt)(a - a_prev) + Kc a + sum of element parts y - f for the columns in
// state `want`; partials of ||R||^2 and ||a||^2
__global__ void __launch_bounds__(NTB) kn_resid(Step S, int64_t ne, const int32_t* __restrict__ inc_ptr,
                                                const int32_t* __restrict__ inc_src, const double* __restrict__ y,
                                                const double* a, const double* aprev, const int* __restrict__ state,
                                                int want, double* R, double* part_rr, double* part_aa) {
    const int t = blockIdx.x / S.nrb, rb = blockIdx.x % S.nrb;
    const int lc = threadIdx.x % G, gc = t * G + lc;
    const bool on = state[gc] == want;
    double sg[3] = {0.0, 0.0, 0.0};
    if (on) {
        const int64_t tt = S.t0 + (int64_t)gc * S.tstride;
        for (int q = 0; q < 3; ++q) sg[q] = S.wave[3 * tt + q];
    }
    const double* at = a + (size_t)t * S.n * G + lc;
    const double* pt = aprev + (size_t)t * S.n * G + lc;
    double rr = 0.0, aa = 0.0;
    const int i1 = min(S.n, (rb + 1) * RBS);
    for (int i = rb * RBS + threadIdx.x / G; i < i1; i += NTB / G) {
        if (!on) continue;
        double m = 0.0, kx = 0.0;
        for (int w = 0; w < S.W; ++w) {
            const int64_t q = (int64_t)w * S.n + i;
            const int j = __ldg(S.col + q);
            const double aj = at[(size_t)j * G];
            m += __ldg(S.M64 + q) * (aj - pt[(size_t)j * G]);
            kx += __ldg(S.Kc + q) * aj;
        }
        double nl = 0.0;
        for (int32_t s = __ldg(inc_ptr + i); s < __ldg(inc_ptr + i + 1); ++s) {
            const int32_t src = __ldg(inc_src + s);
            const int64_t e = src / 3, v = src % 3;
            nl += y[(((size_t)t * 3 + v) * ne + e) * G + lc];
        }
        const double f = S.J0 * (sg[0] * S.F[i] + sg[1] * S.F[S.n + i] + sg[2] * S.F[2 * S.n + i]);
        const double ri = m * S.inv_dt + kx + nl - f;
        R[((size_t)t * S.n + i) * G + lc] = ri;
        const double ai = at[(size_t)i * G];
        rr += ri * ri;
        aa += ai * ai;
    }
    partial_col(rr, part_rr);
    partial_col(aa, part_aa);
}

// ||F||^2 at the start iterate.  With a guess, the start is whichever of the
// guess (residual in part_g) and a_prev (residual in part_p) has the smaller
// residual; accept[c] marks the columns that start from a_prev.
__global__ void kn_first_norm(Cols C, const double* part_g, const double* part_p, int nrb, int kpad) {
    for (int c = threadIdx.x; c < kpad; c += blockDim.x) {
        const double rg = col_sum(part_g, nrb, c);
        const double rp = part_p ? col_sum(part_p, nrb, c) : rg;
        const int prev = part_p && rp < rg;
        C.accept[c] = prev;
        C.nr2[c] = prev ? rp : rg;
    }
}

// Jacobian on the ELL pattern: J = M/dt + Kc + sum_contrib w . N_e (columns in state SOLVE)
__global__ void __launch_bounds__(NTB) kn_jac(int64_t nW, int64_t ne, const double* __restrict__ M64,
                                              const double* __restrict__ Kc, double inv_dt,
                                              const int32_t* __restrict__ jc_ptr, const int32_t* __restrict__ jc_e,
                                              const double* __restrict__ jc_w, const double* __restrict__ N,
                                              double* J64, float* J32, const int* __restrict__ state) {
    const int t = blockIdx.y;
    const int lc = threadIdx.x % G;
    const int64_t q = (int64_t)blockIdx.x * (NTB / G) + threadIdx.x / G;
    if (q >= nW || state[t * G + lc] != ST_SOLVE) return;
    double v = __ldg(M64 + q) * inv_dt + __ldg(Kc + q);
    const size_t vs = (size_t)ne * G;
    for (int32_t s = __ldg(jc_ptr + q); s < __ldg(jc_ptr + q + 1); ++s) {
        const int64_t e = __ldg(jc_e + s);
        const size_t b = ((size_t)t * 3 * ne + e) * G + lc;
        v += __ldg(jc_w + 3 * s) * N[b] + __ldg(jc_w + 3 * s + 1) * N[b + vs] + __ldg(jc_w + 3 * s + 2) * N[b + 2 * vs];
    }
    const size_t o = ((size_t)t * nW + q) * G + lc;
    J64[o] = v;
    J32[o] = (float)v;
}

// coarse operator: Jc = P^T J P per column through the static Galerkin map
__global__ void __launch_bounds__(NTB) kn_galerkin(int64_t nWc, int64_t nWf, const int32_t* __restrict__ gptr,
                                                   const int32_t* __restrict__ gsrc, const double* __restrict__ gw,
                                                   const double* Jf, double* Jc, float* Jc32,
                                                   const int* __restrict__ state) {
    const int t = blockIdx.y;
    const int lc = threadIdx.x % G;
    const int64_t q = (int64_t)blockIdx.x * (NTB / G) + threadIdx.x / G;
    if (q >= nWc || state[t * G + lc] != ST_SOLVE) return;
    double v = 0.0;
    const double* jf = Jf + (size_t)t * nWf * G + lc;
    for (int32_t s = __ldg(gptr + q); s < __ldg(gptr + q + 1); ++s) v += __ldg(gw + s) * jf[(size_t)__ldg(gsrc + s) * G];
    const size_t o = ((size_t)t * nWc + q) * G + lc;
    Jc[o] = v;
    Jc32[o] = (float)v;
}

// 1/diag per row and column, and into *lam the maximum over rows and columns of the
// Gershgorin ratio sum_j |J_ij| / J_ii (rounded up to float; positive floats order
// like their bits, so the maximum is an unsigned atomicMax, one per block)
__global__ void __launch_bounds__(NTB) kn_dinv(int n, int W, int nrb, const int32_t* __restrict__ col,
                                               const double* J64, float* dinv32, int* flag, unsigned* lam,
                                               const int* __restrict__ state) {
    const int t = blockIdx.x / nrb, rb = blockIdx.x % nrb;
    const int lc = threadIdx.x % G;
    const int i1 = min(n, (rb + 1) * RBS);
    const double* jt = J64 + (size_t)t * W * n * G + lc;
    unsigned gmax = 0u;
    const bool on = state[t * G + lc] == ST_SOLVE;  // the bound covers the Jacobians in use
    for (int i = rb * RBS + threadIdx.x / G; on && i < i1; i += NTB / G) {
        double d = 0.0, a = 0.0;
        for (int w = 0; w < W; ++w) {
            const double v = jt[((size_t)w * n + i) * G];
            a += fabs(v);
            if (__ldg(col + w * n + i) == i) d += v;
        }
        if (!(d > 0.0)) {
            atomicExch(flag, 1);
            d = 1.0;
        }
        dinv32[((size_t)t * n + i) * G + lc] = (float)(1.0 / d);
        gmax = max(gmax, __float_as_uint(__double2float_ru(a / d)));
    }
    __shared__ unsigned wmax[NTB / 32];
    gmax = __reduce_max_sync(0xffffffffu, gmax);
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = gmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned m = 0u;
        for (int q = 0; q < NTB / 32; ++q) m = max(m, wmax[q]);
        atomicMax(lam, m);
    }
}

// LD32 = J32 . diag(1/d) of the neighbour row, per column
__global__ void __launch_bounds__(NTB) kn_ld(int64_t nW, int n, const int32_t* __restrict__ col, const float* J32,
                                             const float* dinv32, float* LD32, const int* __restrict__ state) {
    const int t = blockIdx.y;
    const int lc = threadIdx.x % G;
    const int64_t q = (int64_t)blockIdx.x * (NTB / G) + threadIdx.x / G;
    if (q >= nW || state[t * G + lc] != ST_SOLVE) return;
    const int j = __ldg(col + q);
    const size_t o = ((size_t)t * nW + q) * G + lc;
    LD32[o] = J32[o] * dinv32[((size_t)t * n + j) * G + lc];
}

// Banded Cholesky J = L L^T (FP64) of one column per warp, right-looking over a
// ring of u + 1 rows in shared memory (ring row of i: i mod (u+1), entry k holds
// the value at column i - k).  Output in the layout of the banded solve: row i of
// Lb holds 1/L[i][i] at k = 0 and L[i][i-k] at k = 1..u; row i of Ub holds
// 1/L[i][i] at k = 0 and L[i+k][i] at k = 1..u (entries beyond the matrix are
// never read).
__global__ void __launch_bounds__(32) kn_band_factor(int n, int W, int u, int stride, const int32_t* __restrict__ col,
                                                     const double* J64, float* Lb, float* Ub, int* flag,
                                                     const int* __restrict__ state) {
    extern __shared__ double win[];
    const int gc = blockIdx.x, t = gc / G, l = gc % G, lane = threadIdx.x;
    if (state[gc] != ST_SOLVE) return;  // no new Jacobian for this column
    const int U1 = u + 1;
    const double* jt = J64 + (size_t)t * W * n * G + l;
    float* lb = Lb + (size_t)gc * n * stride;
    float* ub = Ub + (size_t)gc * n * stride;
    auto load_row = [&](int i) {
        double* r = win + (size_t)(i % U1) * U1;
        for (int k = lane; k < U1; k += 32) r[k] = 0.0;
        __syncwarp();
        for (int w = lane; w < W; w += 32) {
            const int j = __ldg(col + w * n + i);
            const double v = jt[((size_t)w * n + i) * G];
            // padding entries reference the row itself with value 0
            if (j <= i && i - j <= u && v != 0.0) r[i - j] = v;
        }
        __syncwarp();
    };
    for (int i = 0; i < min(U1, n); ++i) load_row(i);
    for (int j = 0; j < n; ++j) {
        double* rj = win + (size_t)(j % U1) * U1;
        double d = rj[0];
        if (!(d > 0.0)) {
            if (lane == 0) atomicExch(flag, 1);
            d = 1.0;
        }
        d = sqrt(d);
        const double dinv = 1.0 / d;
        const int pmax = min(u, n - 1 - j);
        __syncwarp();
        for (int p = 1 + lane; p <= pmax; p += 32) win[(size_t)((j + p) % U1) * U1 + p] *= dinv;
        __syncwarp();
        for (int p = 1 + lane; p <= pmax; p += 32) {
            double* ri = win + (size_t)((j + p) % U1) * U1;
            const double lij = ri[p];
            for (int q = 1; q <= p; ++q) ri[p - q] -= lij * win[(size_t)((j + q) % U1) * U1 + q];
        }
        __syncwarp();
        for (int k = lane; k <= u; k += 32) {
            if (k == 0) {
                lb[(size_t)j * stride] = (float)dinv;
                ub[(size_t)j * stride] = (float)dinv;
            } else {
                lb[(size_t)j * stride + k] = k <= j ? (float)rj[k] : 0.0f;
                if (k <= j) ub[(size_t)(j - k) * stride + k] = (float)rj[k];
            }
        }
        __syncwarp();
        if (j + U1 < n) load_row(j + U1);
    }
}

// columns needing a direction enter the step-length search with step 1
__global__ void kn_begin_trial(Cols C, int kpad) {
    for (int c = threadIdx.x; c < kpad; c += blockDim.x)
        if (C.state[c] == ST_SOLVE) {
            C.state[c] = ST_TRIAL;
            C.step[c] = 1.0;
            C.halv[c] = 0;
            C.first[c] = 1;
        }
}

// trial point a_t = a + step delta; partial ||delta||^2
__global__ void __launch_bounds__(NTB) kn_trial(int n, int nrb, const double* a, const double* delta, const Cols C,
                                                double* at, double* part_dd) {
    const int t = blockIdx.x / nrb, rb = blockIdx.x % nrb;
    const int lc = threadIdx.x % G, gc = t * G + lc;
    const bool on = C.state[gc] == ST_TRIAL;
    const double st = C.step[gc];
    double dd = 0.0;
    const int i1 = min(n, (rb + 1) * RBS);
    for (int i = rb * RBS + threadIdx.x / G; i < i1; i += NTB / G) {
        if (!on) continue;
        const size_t o = ((size_t)t * n + i) * G + lc;
        const double d = delta[o];
        at[o] = a[o] + st * d;
        dd += d * d;
    }
    partial_col(dd, part_dd);
}

// step-length decisions of one round
__global__ void kn_decide(Cols C, const double* part_rr, const double* part_aa, const double* part_dd, int nrb,
                          int kpad, double tol2, int max_newton, int max_halvings) {
    int trial = 0, solve = 0, its = 0;
    for (int c = threadIdx.x; c < kpad; c += blockDim.x) {
        int acc = 0;
        if (C.state[c] == ST_TRIAL) {
            const double rr = col_sum(part_rr, nrb, c), aa = col_sum(part_aa, nrb, c);
            const double dd = col_sum(part_dd, nrb, c);
            if (C.first[c] && dd <= tol2 * aa) {  // converged: the full correction is taken
                acc = 1;
                C.its[c] += 1;
                C.state[c] = ST_IDLE;
            } else if (rr <= C.nr2[c]) {
                acc = 1;
                C.its[c] += 1;
                C.nr2[c] = rr;
                C.state[c] = C.its[c] >= max_newton ? ST_FAILED : ST_SOLVE;
            } else if (C.halv[c] < max_halvings) {
                C.halv[c] += 1;
                C.step[c] *= 0.5;
                C.first[c] = 0;
            } else {
                C.state[c] = ST_FAILED;
            }
        }
        C.accept[c] = acc;
        trial |= C.state[c] == ST_TRIAL;
        solve |= C.state[c] == ST_SOLVE;
        its += C.its[c];
    }
    trial = __syncthreads_or(trial);
    solve = __syncthreads_or(solve);
    __shared__ int sum;
    if (threadIdx.x == 0) sum = 0;
    __syncthreads();
    atomicAdd(&sum, its);
    __syncthreads();
    if (threadIdx.x == 0) {
        C.flags[0] = trial;
        C.flags[1] = solve;
        C.flags[2] = sum;
    }
}

// accepted columns: a <- a_t, R <- R_t
__global__ void __launch_bounds__(NTB) kn_accept(int n, int nrb, const int* __restrict__ accept, double* a,
                                                 const double* at, double* R, const double* Rt) {
    const int t = blockIdx.x / nrb, rb = blockIdx.x % nrb;
    const int lc = threadIdx.x % G, gc = t * G + lc;
    if (!accept[gc]) return;
    const int i1 = min(n, (rb + 1) * RBS);
    for (int i = rb * RBS + threadIdx.x / G; i < i1; i += NTB / G) {
        const size_t o = ((size_t)t * n + i) * G + lc;
        a[o] = at[o];
        R[o] = Rt[o];
    }
}

// x_out = a + g; failed columns report MG_ENEWTON
__global__ void __launch_bounds__(NTB) kn_out(int n, int nrb, int k, const double* a, const double* __restrict__ g,
                                              int64_t ld_g, double* xout, int64_t ld_out, const int* state,
                                              int* worst) {
    const int t = blockIdx.x / nrb, rb = blockIdx.x % nrb;
    const int lc = threadIdx.x % G, gc = t * G + lc;
    if (gc >= k) return;
    if (rb == 0 && threadIdx.x / G == 0 && state[gc] != ST_IDLE) atomicMin(worst, (int)MG_ENEWTON);
    const int i1 = min(n, (rb + 1) * RBS);
    for (int i = rb * RBS + threadIdx.x / G; i < i1; i += NTB / G) {
        double v = a[((size_t)t * n + i) * G + lc];
        if (g) v += g[(int64_t)i * ld_g + gc];
        xout[(int64_t)i * ld_out + gc] = v;
    }
}

// static set-up kernels
__global__ void kn_jc_weights(int64_t nc, const int32_t* __restrict__ jc_e, const int32_t* __restrict__ jc_ab,
                              const int32_t* __restrict__ eid, const double* __restrict__ grad, double* jc_w) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nc) return;
    const double* g = grad + 6 * (int64_t)eid[jc_e[s]];
    const int a = jc_ab[s] / 3, b = jc_ab[s] % 3;
    jc_w[3 * s] = g[2 * a] * g[2 * b];
    jc_w[3 * s + 1] = g[2 * a] * g[2 * b + 1] + g[2 * a + 1] * g[2 * b];
    jc_w[3 * s + 2] = g[2 * a + 1] * g[2 * b + 1];
}

// ELL stiffness of the linear-law elements
__global__ void kn_kc(int64_t nW, const int32_t* __restrict__ slot, const int32_t* __restrict__ sptr,
                      const int32_t* __restrict__ ssrc, const int32_t* __restrict__ law,
                      const double* __restrict__ elemK, double* Kc) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nW) return;
    const int32_t s = slot[q];
    double v = 0.0;
    if (s >= 0)
        for (int32_t p = sptr[s]; p < sptr[s + 1]; ++p) {
            const int32_t src = ssrc[p];
            if (law[src / 9] == 0) v += elemK[src];
        }
    Kc[q] = v;
}

}  // namespace

// ------------------------------------------------------------------ static data

bool mesh_is_nonlinear(const mg_ctx* c, int mesh) { return c->meshes[mesh].n_nl > 0; }

// parent dofs and weights of each fine dof (<= 2), as in the prolongation
static void parent_weights(const mg_ctx* c, int fine, std::vector<int32_t>& par, std::vector<double>& pw) {
    const MeshLevel& mf = c->meshes[fine];
    const MeshLevel& mc = c->meshes[mf.parent_mesh];
    const std::vector<int32_t>* parent = nullptr;
    for (auto& r : c->refinements)
        if (r.first.first == fine && r.first.second == mf.parent_mesh) parent = &r.second;
    if (!parent) mg_fail(MG_ESTATE, "refinement of a multigrid depth not found");
    par.assign(2 * mf.n, -1);
    pw.assign(2 * mf.n, 0.0);
    for (int64_t i = 0; i < mf.n; ++i) {
        const int32_t v = mf.dof2node[i];
        const int32_t a = (*parent)[2 * v], b = (*parent)[2 * v + 1];
        if (a == b) {
            par[i] = mc.node2dof[a];
            pw[i] = 1.0;
        } else {
            par[i] = mc.node2dof[a];
            par[mf.n + i] = mc.node2dof[b];
            pw[i] = 0.5;
            pw[mf.n + i] = 0.5;
        }
        for (int q = 0; q < 2; ++q)
            if (par[q * mf.n + i] < 0) pw[q * mf.n + i] = 0.0;
    }
}

// ELL position of column j in row i of mesh m (host CSR), or -1
static int ell_pos(const MeshLevel& m, int32_t i, int32_t j) {
    auto b = m.col_h.begin() + m.rowptr_h[i], e = m.col_h.begin() + m.rowptr_h[i + 1];
    auto it = std::lower_bound(b, e, j);
    return (it != e && *it == j) ? (int)(it - b) : -1;
}

static void csr_from_pairs(int64_t rows, const std::vector<std::pair<int64_t, int64_t>>& key_idx,
                           std::vector<int32_t>& ptr, std::vector<int32_t>& order) {
    ptr.assign(rows + 1, 0);
    for (auto& p : key_idx) ptr[p.first + 1]++;
    std::partial_sum(ptr.begin(), ptr.end(), ptr.begin());
    order.assign(key_idx.size(), 0);
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (auto& p : key_idx) order[fill[p.first]++] = (int32_t)p.second;
}

static NlMesh& nl_mesh(mg_ctx* c, int mesh) {
    auto it = c->nl.find(mesh);
    if (it != c->nl.end()) return *it->second;
    auto* N = new NlMesh();
    c->nl[mesh] = N;
    N->mesh = mesh;
    MeshLevel& m = c->meshes[mesh];
    const int64_t n = m.n, W = m.ell_W, nW = W * n;
    cudaStream_t s = c->stream;
    // bandwidth
    int u = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int32_t q = m.rowptr_h[i]; q < m.rowptr_h[i + 1]; ++q) u = std::max(u, (int)std::abs(m.col_h[q] - (int)i));
    N->band_u = u;
    N->band_stride = (u + 1 + 3) / 4 * 4;
    // nonlinear elements
    std::vector<int32_t> eid, edof;
    for (int64_t e = 0; e < m.n_tri; ++e)
        if (c->mats[m.region[e]].law == 1) {
            eid.push_back((int32_t)e);
            for (int v = 0; v < 3; ++v) edof.push_back(m.node2dof[m.tri[3 * e + v]]);
        }
    N->ne = (int64_t)eid.size();
    upload(N->eid, eid);
    upload(N->edof, edof);
    // dof -> (nonlinear element, vertex)
    std::vector<std::pair<int64_t, int64_t>> inc;
    for (int64_t e = 0; e < N->ne; ++e)
        for (int v = 0; v < 3; ++v)
            if (edof[3 * e + v] >= 0) inc.push_back({edof[3 * e + v], 3 * e + v});
    std::vector<int32_t> ptr, ord;
    csr_from_pairs(n, inc, ptr, ord);
    upload(N->inc_ptr, ptr);
    upload(N->inc_src, ord);
    // ELL entry -> (nonlinear element, local a, b)
    std::vector<std::pair<int64_t, int64_t>> jc;
    for (int64_t e = 0; e < N->ne; ++e)
        for (int a = 0; a < 3; ++a) {
            const int32_t da = edof[3 * e + a];
            if (da < 0) continue;
            for (int b = 0; b < 3; ++b) {
                const int32_t db = edof[3 * e + b];
                if (db < 0) continue;
                const int w = ell_pos(m, da, db);
                jc.push_back({(int64_t)w * n + da, 9 * e + 3 * a + b});
            }
        }
    csr_from_pairs(nW, jc, ptr, ord);
    std::vector<int32_t> jce(ord.size()), jcab(ord.size());
    for (size_t q = 0; q < ord.size(); ++q) {
        jce[q] = ord[q] / 9;
        jcab[q] = ord[q] % 9;
    }
    upload(N->jc_ptr, ptr);
    upload(N->jc_e, jce);
    DBuf ab;
    upload(ab, jcab);
    N->jc_w.ensure(std::max<size_t>(1, 3 * jce.size()) * sizeof(double));
    if (!jce.empty())
        kn_jc_weights<<<nblk((int64_t)jce.size()), NTB, 0, s>>>((int64_t)jce.size(), N->jc_e.as<int32_t>(),
                                                               ab.as<int32_t>(), N->eid.as<int32_t>(),
                                                               m.grad.as<double>(), N->jc_w.as<double>());
    N->Kc.ensure(nW * sizeof(double));
    kn_kc<<<nblk(nW), NTB, 0, s>>>(nW, m.ell_slot.as<int32_t>(), m.slot_ptr.as<int32_t>(), m.slot_src.as<int32_t>(),
                                   m.elem_law.as<int32_t>(), m.elemK.as<double>(), N->Kc.as<double>());
    // Galerkin map onto the parent mesh: coarse entry (I, J) += w_iI w_jJ J[i, j]
    if (m.parent_mesh >= 0) {
        const MeshLevel& mc = c->meshes[m.parent_mesh];
        std::vector<int32_t> par;
        std::vector<double> pw;
        parent_weights(c, mesh, par, pw);
        std::vector<std::pair<int64_t, int64_t>> gl;  // (coarse ELL entry, contribution)
        std::vector<int32_t> fsrc;                      // fine ELL entry of each contribution
        std::vector<double> gwv;                        // its weight
        for (int64_t i = 0; i < n; ++i)
            for (int32_t q = m.rowptr_h[i]; q < m.rowptr_h[i + 1]; ++q) {
                const int32_t j = m.col_h[q];
                const int64_t fq = (int64_t)(q - m.rowptr_h[i]) * n + i;
                for (int x = 0; x < 2; ++x)
                    for (int y = 0; y < 2; ++y) {
                        const int32_t I = par[x * n + i], J = par[y * n + j];
                        if (I < 0 || J < 0) continue;
                        const int w = ell_pos(mc, I, J);
                        if (w < 0) mg_fail(MG_EINVAL, "Galerkin product leaves the coarse pattern (meshes not nested)");
                        gl.push_back({(int64_t)w * mc.n + I, (int64_t)gwv.size()});
                        fsrc.push_back((int32_t)fq);
                        gwv.push_back(pw[x * n + i] * pw[y * n + j]);
                    }
            }
        csr_from_pairs((int64_t)mc.ell_W * mc.n, gl, ptr, ord);
        std::vector<int32_t> src(ord.size());
        std::vector<double> wv(ord.size());
        for (size_t q = 0; q < ord.size(); ++q) {
            src[q] = fsrc[ord[q]];
            wv[q] = gwv[ord[q]];
        }
        upload(N->gal_ptr, ptr);
        upload(N->gal_src, src);
        upload(N->gal_w, wv);
    }
    MG_CUDA(cudaGetLastError());
    return *N;
}

// ------------------------------------------------------------------ plan

struct NewtonPlan {
    const StepOp* op = nullptr;
    int ntile = 0;
    std::vector<DBuf> bufs;
    double *a = nullptr, *aprev = nullptr, *at = nullptr, *R = nullptr, *Rt = nullptr, *yN = nullptr;
    double* part = nullptr;  // 3 partial arrays
    PcOperator pco{};
    double* J64[MG_MAX_DEPTH] = {};
    Cols cols{};
    int* flags_h = nullptr;  // pinned
    GraphPlan* pcg = nullptr;
    mg_solver_opts pso{};  // options the PCG graph was built with
    unsigned* lam = nullptr;  // per depth: Gershgorin bound of the current Jacobians
    std::vector<int> mesh_of_depth;
    ~NewtonPlan() {
        if (pcg) graph_plan_delete(pcg);
        if (flags_h) cudaFreeHost(flags_h);
    }
};

void newton_plan_delete(NewtonPlan* p) { delete p; }

static void* nalloc(NewtonPlan& P, cudaStream_t s, size_t bytes) {
    P.bufs.emplace_back();
    P.bufs.back().ensure(bytes);
    MG_CUDA(cudaMemsetAsync(P.bufs.back().p, 0, bytes, s));
    return P.bufs.back().p;
}

// the options the correction's PCG graph depends on
static bool same_pcg_shape(const mg_solver_opts& a, const mg_solver_opts& b) {
    return smooth_sweeps(a) == smooth_sweeps(b) && a.omega == b.omega && a.smoother == b.smoother &&
           a.cheb_ratio == b.cheb_ratio && a.rows_per_block == b.rows_per_block &&
           a.coarse_rows_per_block == b.coarse_rows_per_block && a.base_tiles == b.base_tiles;
}

static NewtonPlan* newton_plan(mg_ctx* c, const StepOp& op, int ntile, const mg_solver_opts& so) {
    for (auto* p : c->nplans)
        if (p->op == &op && p->ntile == ntile) {
            if (!same_pcg_shape(p->pso, so)) {  // rebuild the correction's graph for new options
                graph_plan_delete(p->pcg);
                p->pcg = nullptr;
                p->pcg = graph_plan_pc(c, op, ntile, so, p->pco);
                p->pso = so;
            }
            return p;
        }
    auto* P = new NewtonPlan();
    cudaStream_t s = c->stream;
    try {
        P->op = &op;
        P->ntile = ntile;
        const int kpad = ntile * G;
        const MeshLevel& m0 = c->meshes[op.mesh];
        const int nd = (int)op.mg.size();
        const size_t e0 = (size_t)kpad * m0.n;
        P->a = (double*)nalloc(*P, s, e0 * 8);
        P->aprev = (double*)nalloc(*P, s, e0 * 8);
        P->at = (double*)nalloc(*P, s, e0 * 8);
        P->R = (double*)nalloc(*P, s, e0 * 8);
        P->Rt = (double*)nalloc(*P, s, e0 * 8);
        NlMesh& N0 = nl_mesh(c, op.mesh);
        P->yN = (double*)nalloc(*P, s, std::max<size_t>(1, (size_t)3 * N0.ne * kpad) * 8);
        const int nrb0 = (int)((m0.n + RBS - 1) / RBS);
        P->part = (double*)nalloc(*P, s, (size_t)3 * ntile * nrb0 * G * 8);
        for (int d = 0; d < nd; ++d) {
            const MeshLevel& md = c->meshes[op.mg[d]->mesh];
            P->mesh_of_depth.push_back(op.mg[d]->mesh);
            const size_t nW = (size_t)md.ell_W * md.n * kpad;
            P->J64[d] = (double*)nalloc(*P, s, nW * 8);
            P->pco.d[d].J64 = P->J64[d];
            P->pco.d[d].J32 = (float*)nalloc(*P, s, nW * 4);
            P->pco.d[d].LD32 = (float*)nalloc(*P, s, nW * 4);
            P->pco.d[d].dinv32 = (float*)nalloc(*P, s, (size_t)md.n * kpad * 4);
            if (d + 1 < nd) nl_mesh(c, op.mg[d]->mesh);  // Galerkin map to the next depth
        }
        const MeshLevel& mb = c->meshes[op.mg[nd - 1]->mesh];
        NlMesh& Nb = nl_mesh(c, op.mg[nd - 1]->mesh);
        if (Nb.band_u >= 128) mg_fail(MG_EINVAL, "base mesh bandwidth above 127: number it with a small bandwidth");
        if (mb.ell_W > 32) mg_fail(MG_EINVAL, "more than 32 neighbours per row in the base mesh");
        P->pco.band_u = Nb.band_u;
        P->pco.band_stride = Nb.band_stride;
        const size_t bsz = (size_t)kpad * mb.n * Nb.band_stride * 4;
        P->pco.band_L = (float*)nalloc(*P, s, bsz);
        P->pco.band_U = (float*)nalloc(*P, s, bsz);
        P->pco.R = P->R;
        char* cb = (char*)nalloc(*P, s, (size_t)kpad * (5 * 4 + 2 * 8) + 64);
        P->cols.step = (double*)cb;
        P->cols.nr2 = P->cols.step + kpad;
        P->cols.state = (int*)(P->cols.nr2 + kpad);
        P->cols.accept = P->cols.state + kpad;
        P->cols.halv = P->cols.accept + kpad;
        P->cols.its = P->cols.halv + kpad;
        P->cols.first = P->cols.its + kpad;
        P->cols.flags = P->cols.first + kpad;
        P->pco.state = P->cols.state;
        P->lam = (unsigned*)nalloc(*P, s, MG_MAX_DEPTH * sizeof(unsigned));
        P->pco.lam = P->lam;
        MG_CUDA(cudaMallocHost(&P->flags_h, 4 * sizeof(int)));
        MG_CUDA(cudaStreamSynchronize(s));
        P->pcg = graph_plan_pc(c, op, ntile, so, P->pco);
        P->pso = so;
        c->nplans.push_back(P);
        return P;
    } catch (...) {
        delete P;
        throw;
    }
}

// ------------------------------------------------------------------ one batched Newton step

void phi_batch_newton(mg_ctx* c, const StepOp& op, const PhiIO& io, const mg_solver_opts& so,
                      SolveCounters* counters) {
    if (so.precision != MG_FP64 || so.precond != MG_PRECOND_MULTIGRID)
        mg_fail(MG_EINVAL, "nonlinear steps use the FP64 form with the multigrid preconditioner");
    if (!(so.newton_tol > 0.0) || so.max_newton < 1 || so.max_halvings < 0 || !(so.newton_lin_tol > 0.0) ||
        !(so.newton_lin_tol < 1.0))
        mg_fail(MG_EINVAL, "bad Newton options");
    mg_solver_opts lin = so;  // the corrections' PCG stops at newton_lin_tol
    lin.cg_tol = so.newton_lin_tol;
    const int ntile = (io.k + G - 1) / G, kpad = ntile * G;
    NewtonPlan* P = newton_plan(c, op, ntile, so);
    const MeshLevel& m0 = c->meshes[op.mesh];
    NlMesh& N0 = nl_mesh(c, op.mesh);
    const MgDepth& d0 = *op.mg[0];
    cudaStream_t s = c->stream;
    const int nrb0 = (int)((m0.n + RBS - 1) / RBS);
    const unsigned g0 = (unsigned)(ntile * nrb0);
    double* part_rr = P->part;
    double* part_aa = part_rr + (size_t)ntile * nrb0 * G;
    double* part_dd = part_aa + (size_t)ntile * nrb0 * G;
    int64_t launches = 0;
    int rounds = 0, newton_its = 0;
    const auto t_start = std::chrono::steady_clock::now();

    Step S = {};
    S.n = (int)m0.n;
    S.W = m0.ell_W;
    S.nrb = nrb0;
    S.k = io.k;
    S.col = m0.ell_col.as<int32_t>();
    S.M64 = d0.M64.as<double>();
    S.Kc = N0.Kc.as<double>();
    S.F = m0.F.as<double>();
    S.inv_dt = 1.0 / op.dt;
    S.J0 = c->pwm.J0;
    S.wave = io.wave;
    S.t0 = io.t0;
    S.tstride = io.tstride;
    Elems E = {};
    E.ne = N0.ne;
    E.eid = N0.eid.as<int32_t>();
    E.edof = N0.edof.as<int32_t>();
    E.grad = m0.grad.as<double>();
    E.area = m0.area.as<double>();
    E.kk = m0.elem_k.as<double>();
    E.n = (int)m0.n;
    const dim3 ge(std::max<unsigned>(1, nblk(N0.ne, NTB / G)), ntile);
    const double tol2 = so.newton_tol * so.newton_tol;
    c->flag.ensure(sizeof(int) * 4);
    MG_CUDA(cudaMemsetAsync(c->flag.p, 0, sizeof(int), s));

    kn_init<<<g0, NTB, 0, s>>>(S, io.xprev, io.ld_prev, io.guess, io.ld_guess, io.g, io.ld_g, P->a, P->aprev);
    kn_state_init<<<1, 1024, 0, s>>>(P->cols, io.k, kpad);
    kn_elem<0><<<ge, NTB, 0, s>>>(E, P->a, P->cols.state, ST_SOLVE, P->yN);
    kn_resid<<<g0, NTB, 0, s>>>(S, N0.ne, N0.inc_ptr.as<int32_t>(), N0.inc_src.as<int32_t>(), P->yN, P->a, P->aprev,
                                P->cols.state, ST_SOLVE, P->R, part_rr, part_aa);
    launches += 4;
    if (io.guess) {
        // residual at a_prev as well: each column starts from the better of the two
        kn_elem<0><<<ge, NTB, 0, s>>>(E, P->aprev, P->cols.state, ST_SOLVE, P->yN);
        kn_resid<<<g0, NTB, 0, s>>>(S, N0.ne, N0.inc_ptr.as<int32_t>(), N0.inc_src.as<int32_t>(), P->yN, P->aprev,
                                    P->aprev, P->cols.state, ST_SOLVE, P->Rt, part_dd, part_aa);
        kn_first_norm<<<1, 1024, 0, s>>>(P->cols, part_rr, part_dd, nrb0, kpad);
        kn_accept<<<g0, NTB, 0, s>>>((int)m0.n, nrb0, P->cols.accept, P->a, P->aprev, P->R, P->Rt);
        launches += 4;
    } else {
        kn_first_norm<<<1, 1024, 0, s>>>(P->cols, part_rr, nullptr, nrb0, kpad);
        launches += 1;
    }
    const int nd = (int)op.mg.size();
    for (int it = 0; it < so.max_newton; ++it) {
        // Jacobian hierarchy of every column at its current iterate
        kn_elem<1><<<ge, NTB, 0, s>>>(E, P->a, P->cols.state, 0, P->yN);
        const int64_t nW0 = (int64_t)m0.ell_W * m0.n;
        kn_jac<<<dim3(nblk(nW0, NTB / G), ntile), NTB, 0, s>>>(nW0, N0.ne, d0.M64.as<double>(), N0.Kc.as<double>(),
                                                               1.0 / op.dt, N0.jc_ptr.as<int32_t>(),
                                                               N0.jc_e.as<int32_t>(), N0.jc_w.as<double>(), P->yN,
                                                               P->J64[0], P->pco.d[0].J32, P->cols.state);
        launches += 2;
        MG_CUDA(cudaMemsetAsync(P->lam, 0, MG_MAX_DEPTH * sizeof(unsigned), s));
        for (int d = 0; d < nd; ++d) {
            const MeshLevel& md = c->meshes[P->mesh_of_depth[d]];
            const int64_t nW = (int64_t)md.ell_W * md.n;
            if (d > 0) {
                const MeshLevel& mf = c->meshes[P->mesh_of_depth[d - 1]];
                NlMesh& Nf = nl_mesh(c, P->mesh_of_depth[d - 1]);
                kn_galerkin<<<dim3(nblk(nW, NTB / G), ntile), NTB, 0, s>>>(
                    nW, (int64_t)mf.ell_W * mf.n, Nf.gal_ptr.as<int32_t>(), Nf.gal_src.as<int32_t>(),
                    Nf.gal_w.as<double>(), P->J64[d - 1], P->J64[d], P->pco.d[d].J32, P->cols.state);
                launches += 1;
            }
            const int nrb = (int)((md.n + RBS - 1) / RBS);
            kn_dinv<<<ntile * nrb, NTB, 0, s>>>((int)md.n, md.ell_W, nrb, md.ell_col.as<int32_t>(), P->J64[d],
                                                P->pco.d[d].dinv32, c->flag.as<int>(), P->lam + d, P->cols.state);
            kn_ld<<<dim3(nblk(nW, NTB / G), ntile), NTB, 0, s>>>(nW, (int)md.n, md.ell_col.as<int32_t>(),
                                                                 P->pco.d[d].J32, P->pco.d[d].dinv32,
                                                                 P->pco.d[d].LD32, P->cols.state);
            launches += 2;
        }
        {
            const MeshLevel& mb = c->meshes[P->mesh_of_depth[nd - 1]];
            const int u = P->pco.band_u;
            const size_t smem = (size_t)(u + 1) * (u + 1) * sizeof(double);
            if (smem > 48 * 1024)
                MG_CUDA(cudaFuncSetAttribute(kn_band_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kn_band_factor<<<kpad, 32, smem, s>>>((int)mb.n, mb.ell_W, u, P->pco.band_stride,
                                                  mb.ell_col.as<int32_t>(), P->J64[nd - 1],
                                                  const_cast<float*>(P->pco.band_L), const_cast<float*>(P->pco.band_U),
                                                  c->flag.as<int>(), P->cols.state);
            launches += 1;
        }
        // Newton correction of the columns in state SOLVE
        graph_plan_run(c, P->pcg, io.k, lin);
        launches += 1;
        const double* delta = graph_plan_solution(P->pcg);
        kn_begin_trial<<<1, 1024, 0, s>>>(P->cols, kpad);
        launches += 1;
        bool more = false;
        ++newton_its;
        for (int h = 0; h <= so.max_halvings; ++h) {
            ++rounds;
            kn_trial<<<g0, NTB, 0, s>>>((int)m0.n, nrb0, P->a, delta, P->cols, P->at, part_dd);
            kn_elem<0><<<ge, NTB, 0, s>>>(E, P->at, P->cols.state, ST_TRIAL, P->yN);
            kn_resid<<<g0, NTB, 0, s>>>(S, N0.ne, N0.inc_ptr.as<int32_t>(), N0.inc_src.as<int32_t>(), P->yN, P->at,
                                        P->aprev, P->cols.state, ST_TRIAL, P->Rt, part_rr, part_aa);
            kn_decide<<<1, 1024, 0, s>>>(P->cols, part_rr, part_aa, part_dd, nrb0, kpad, tol2, so.max_newton,
                                         so.max_halvings);
            kn_accept<<<g0, NTB, 0, s>>>((int)m0.n, nrb0, P->cols.accept, P->a, P->at, P->R, P->Rt);
            launches += 5;
            MG_CUDA(cudaMemcpyAsync(P->flags_h, P->cols.flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
            MG_CUDA(cudaStreamSynchronize(s));
            more = P->flags_h[1] != 0;
            if (!P->flags_h[0]) break;
        }
        if (!more) break;
    }
    kn_out<<<g0, NTB, 0, s>>>((int)m0.n, nrb0, io.k, P->a, io.g, io.ld_g, io.xout, io.ld_out, P->cols.state,
                              (int*)((char*)c->counters.p + 8));
    launches += 1;
    MG_CUDA(cudaGetLastError());
    int bad = 0;
    MG_CUDA(cudaMemcpyAsync(&bad, c->flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    if (bad) mg_fail(MG_ENEWTON, "Newton Jacobian lost positive definiteness (non-finite iterate)");
    if (mg_trace_level() >= 2) {
        const double ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        std::fprintf(stderr, "[newton] mesh %d  k %d  iterations %d  rounds %d  column-iterations %d  %.1f ms\n",
                     op.mesh, io.k, newton_its, rounds, P->flags_h[2], ms);
    }
    if (counters) {
        counters->step_solves += io.k;
        counters->batched_steps += 1;
        counters->launches += launches;
        counters->newton_iters += P->flags_h[2];
    }
}
