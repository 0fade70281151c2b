// FAS-MGRIT driver (Algorithm 1, Sec. 2.1-2.2) and sequential stepping (Sec. 2).
//
// Storage of one non-coarsest time level l with N_l intervals and factor m:
// m "slabs", slab j holding the points t = c*m + j (c = 0..N_l/m) as the columns
// of a node-major n_l x ld matrix (ld >= N_l/m + 1).  F-relaxation step j then
// reads slab j-1 and writes slab j, C-relaxation reads slab m-1 and writes slab 0
// shifted by one column: every batched step works on unit-stride columns.  The
// coarsest level stores its points time-major and is solved sequentially.
//
// One iteration on level l (relaxation, C-point residual r_c = g_cm - u_cm +
// Phi(u_cm-1), restriction by injection in time and R_s in space, FAS right-hand
// side G = A_2(u2) + g2, recursive coarse solve, correction u_cm += P_s(v - u2)
// and, below the finest level, the F-relaxation that completes ideal
// interpolation) follows Algorithm 1; on the finest level that F-relaxation is
// the first step of the next iteration's relaxation, which computes the same
// values.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <set>
#include <vector>

#include "internal.h"

namespace {

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Address of (time point t, node i) of a level store.
struct LevelView {
    double* base;
    int64_t n, m, ld, slab;  // m == 0: time-major
    __host__ __device__ int64_t idx(int64_t t, int64_t i) const {
        if (m == 0) return t * n + i;
        return (t % m) * slab + i * ld + t / m;
    }
};

// r[i][c] = g(cm) - u(cm) + V[i][c-1] for c >= 1, r[i][0] = 0; partial sums of r^2.
__global__ void k_cpoint_residual(int64_t n, int64_t NT, const double* __restrict__ U0, const double* __restrict__ G0,
                                  int64_t ld, const double* __restrict__ V, int64_t ldv, double* __restrict__ R,
                                  int64_t ldr, double* __restrict__ partial) {
    __shared__ double red[256];
    double acc = 0.0;
    const int64_t total = n * (NT + 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / (NT + 1), c = q % (NT + 1);
        double r = 0.0;
        if (c > 0) {
            r = V[i * ldv + c - 1] - U0[i * ld + c];
            if (G0) r += G0[i * ld + c];
        }
        R[i * ldr + c] = r;
        acc += r * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(int nb, const double* __restrict__ partial, double* __restrict__ out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) acc += partial[q];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// Restriction (Algorithm 1, restriction step): W[:, c] = R_s u(cm) (injection at coarse
// nodes), g2[:, c] = R_s r_c with mode 0 injection, 1 P^T, 2 diag(P^T 1)^-1 P^T.
__global__ void k_restrict(int64_t nc, int64_t NT, const double* __restrict__ U0, int64_t ld,
                           const double* __restrict__ R, int64_t ldr, const int32_t* __restrict__ inj,
                           const int32_t* __restrict__ pt_ptr, const int32_t* __restrict__ pt_col,
                           const double* __restrict__ pt_val, const double* __restrict__ rinv, int mode,
                           double* __restrict__ W, double* __restrict__ g2, int64_t ldw) {
    const int64_t total = nc * (NT + 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t ic = q / (NT + 1), c = q % (NT + 1);
        int64_t src = inj ? inj[ic] : ic;
        W[ic * ldw + c] = U0[src * ld + c];
        double gv;
        if (!inj || mode == 0) {
            gv = R[src * ldr + c];
        } else {
            gv = 0.0;
            for (int32_t e = pt_ptr[ic]; e < pt_ptr[ic + 1]; ++e) gv += pt_val[e] * R[(int64_t)pt_col[e] * ldr + c];
            if (mode == 2) gv *= rinv[ic];
        }
        g2[ic * ldw + c] = gv;
    }
}

// FAS right-hand side of the coarse level (Algorithm 1, coarse problem):
// G_0 = u2_0 + g2_0, G_c = u2_c - Phi_c(u2_{c-1}) + g2_c; coarse iterate v = u2.
__global__ void k_fas_rhs(int64_t nc, int64_t Nc, const double* __restrict__ W, const double* __restrict__ g2,
                          const double* __restrict__ Vc, int64_t ldw, LevelView Gv, LevelView Uv) {
    const int64_t total = nc * (Nc + 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / (Nc + 1), t = q % (Nc + 1);
        double w = W[i * ldw + t];
        double gval = w + g2[i * ldw + t];
        if (t > 0) gval -= Vc[i * ldw + t - 1];
        Gv.base[Gv.idx(t, i)] = gval;
        Uv.base[Uv.idx(t, i)] = w;
    }
}

// Correction (Algorithm 1, coarse-grid correction): u(cm) += P_s (v_c - u2_c), c = 1..NT.
__global__ void k_correct(int64_t nf, int64_t NT, double* __restrict__ U0, int64_t ld, LevelView Vv,
                          const double* __restrict__ W, int64_t ldw, const int32_t* __restrict__ p_ptr,
                          const int32_t* __restrict__ p_col, const double* __restrict__ p_val) {
    const int64_t total = nf * NT;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / NT, c = q % NT + 1;
        double e;
        if (p_ptr) {
            e = 0.0;
            for (int32_t k = p_ptr[i]; k < p_ptr[i + 1]; ++k) {
                int64_t j = p_col[k];
                e += p_val[k] * (Vv.base[Vv.idx(c, j)] - W[j * ldw + c]);
            }
        } else {
            e = Vv.base[Vv.idx(c, i)] - W[i * ldw + c];
        }
        U0[i * ld + c] += e;
    }
}

// Nested iterations: C-points c = 1..NT of the fine level <- P_s v_c of the coarse
// level's iterate (identity when the meshes agree).
__global__ void k_interp_cpoints(int64_t nf, int64_t NT, LevelView Fv, int64_t m, LevelView Cv,
                                 const int32_t* __restrict__ p_ptr, const int32_t* __restrict__ p_col,
                                 const double* __restrict__ p_val) {
    const int64_t total = nf * NT;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / NT, c = q % NT + 1;
        double v;
        if (p_ptr) {
            v = 0.0;
            for (int32_t k = p_ptr[i]; k < p_ptr[i + 1]; ++k) v += p_val[k] * Cv.base[Cv.idx(c, p_col[k])];
        } else {
            v = Cv.base[Cv.idx(c, i)];
        }
        Fv.base[Fv.idx(c * m, i)] = v;
    }
}

// dst[j] = src[inj[j]] (nodal injection of a state), or a copy without inj
__global__ void k_gather_state(int64_t nc, const int32_t* __restrict__ inj, const double* __restrict__ src,
                               double* __restrict__ dst) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < nc) dst[j] = src[inj ? inj[j] : j];
}

// Joule losses (Eq. losses, per unit depth): P = d^T M_sigma d with d = (u_t - u_{t-1}) / dt.
// One block per time point; UV gives u_t, PV u_{t-1}; a fixed-order block sum.
__device__ void joule_block(int64_t n, LevelView Uv, int64_t t, int64_t tp, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ col, const double* __restrict__ M, double inv_dt,
                            double* out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double dr = (Uv.base[Uv.idx(t, r)] - Uv.base[Uv.idx(tp, r)]) * inv_dt;
        double md = 0.0;
        for (int32_t k = rp[r]; k < rp[r + 1]; ++k) {
            const int64_t j = col[k];
            md += M[k] * ((Uv.base[Uv.idx(t, j)] - Uv.base[Uv.idx(tp, j)]) * inv_dt);
        }
        acc += dr * md;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// losses at every time point of a trajectory (block t-1 -> point t, t = 1..N)
__global__ void k_joule_traj(int64_t n, LevelView Uv, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const double* __restrict__ M, double inv_dt, double* out) {
    const int64_t t = blockIdx.x + 1;
    joule_block(n, Uv, t, t - 1, rp, col, M, inv_dt, out + t);
}

// losses at the C-points c = 1..NT of a level store (point cm from cm-1)
__global__ void k_joule_cpoints(int64_t n, LevelView Uv, int64_t m, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const double* __restrict__ M, double inv_dt,
                                double* out) {
    const int64_t c = blockIdx.x + 1;
    joule_block(n, Uv, c * m, c * m - 1, rp, col, M, inv_dt, out + c);
}

// max_c |P_new - P_old| / |P_new| into *res (infinite on the first call), then P_old = P_new
__global__ void k_joule_change(int64_t NT, const double* __restrict__ pnew, double* __restrict__ pold, int first,
                               double* res) {
    __shared__ double red[256];
    double mx = 0.0;
    for (int64_t c = 1 + threadIdx.x; c <= NT; c += blockDim.x) {
        const double a = pnew[c], b = pold[c];
        const double den = a != 0.0 ? fabs(a) : 1.0;
        mx = fmax(mx, fabs(a - b) / den);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *res = first ? INFINITY : red[0];
    __syncthreads();
    for (int64_t c = threadIdx.x; c <= NT; c += blockDim.x) pold[c] = pnew[c];
}

// Level store -> time-major trajectory.
__global__ void k_to_time_major(int64_t n, int64_t N, LevelView Uv, double* __restrict__ out) {
    const int64_t total = n * (N + 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t t = q / n, i = q % n;
        out[q] = Uv.base[Uv.idx(t, i)];
    }
}

__global__ void k_fill_column(int64_t n, const double* __restrict__ src, double* __restrict__ dst, int64_t ld) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i * ld] = src[i];
}

struct Level {
    int mesh = 0;
    int64_t n = 0, N = 0, m = 0, NT = 0, ld = 0, stride = 1;
    double dt = 0.0;
    StepOp* op = nullptr;
    Transfer* tr = nullptr;  // to the next level (null if the same mesh)
    double *U = nullptr, *G = nullptr;     // iterate and FAS right-hand side (G null on level 0)
    double *R = nullptr, *V = nullptr;     // C-point residual and Phi(u_cm-1) (n x ld)
    double *W = nullptr, *g2 = nullptr, *Vc = nullptr;  // restricted state / residual / coarse Phi (this level's mesh)
    int64_t ldw = 0;
    LevelView view() const { return LevelView{U, n, m, ld, n * ld}; }
    LevelView gview() const { return LevelView{G, n, m, ld, n * ld}; }
};

struct Solver {
    mg_ctx* c;
    int64_t N;
    double T;
    mg_opts o;
    std::vector<Level> lv;
    const double* wave = nullptr;      // source waveform of the iterations (PWM, with the ramp)
    const double* wave_ref = nullptr;  // sine reference (nested iterations with nested == 2)
    SolveCounters cnt;
    double* partial = nullptr;
    double* norm = nullptr;
    static constexpr int kRedBlocks = 304;

    void phi(int l, int k, const double* xprev, int64_t ldp, double* xout, int64_t ldo, const double* g,
             int64_t ldg, int64_t t0, int64_t tstride) {
        PhiIO io;
        io.k = k;
        io.xprev = xprev;
        io.ld_prev = ldp;
        io.g = g;
        io.ld_g = ldg;
        io.guess = xout;  // warm start from the current iterate
        io.ld_guess = ldo;
        io.xout = xout;
        io.ld_out = ldo;
        io.wave = wave;
        io.t0 = t0;
        io.tstride = tstride;
        phi_batch(c, *lv[l].op, io, o.solver, &cnt);
    }

    // F-relaxation: u(cm+j) = Phi(u(cm+j-1)) + g(cm+j), j = 1..m-1, all intervals at once.
    void f_relax(int l) {
        Level& L = lv[l];
        const int64_t slab = L.n * L.ld;
        for (int64_t j = 1; j < L.m; ++j)
            phi(l, (int)L.NT, L.U + (j - 1) * slab, L.ld, L.U + j * slab, L.ld, L.G ? L.G + j * slab : nullptr, L.ld,
                j * L.stride, L.m * L.stride);
    }

    // C-relaxation: u(cm) = Phi(u(cm-1)) + g(cm), c = 1..NT.
    void c_relax(int l) {
        Level& L = lv[l];
        const int64_t slab = L.n * L.ld;
        phi(l, (int)L.NT, L.U + (L.m - 1) * slab, L.ld, L.U + 1, L.ld, L.G ? L.G + 1 : nullptr, L.ld,
            L.m * L.stride, L.m * L.stride);
    }

    void relax(int l) {
        f_relax(l);
        for (int q = 0; q < o.relax; ++q) {
            c_relax(l);
            f_relax(l);
        }
    }

    // r_c for c = 0..NT into L.R; if want_norm, the squared norm into norm[0].
    void residual(int l) {
        Level& L = lv[l];
        const int64_t slab = L.n * L.ld;
        PhiIO io;
        io.k = (int)L.NT;
        io.xprev = L.U + (L.m - 1) * slab;
        io.ld_prev = L.ld;
        io.guess = L.U + 1;  // Phi(u(cm-1)) is close to u(cm)
        io.ld_guess = L.ld;
        io.xout = L.V;
        io.ld_out = L.ld;
        io.wave = wave;
        io.t0 = L.m * L.stride;
        io.tstride = L.m * L.stride;
        phi_batch(c, *L.op, io, o.solver, &cnt);
        k_cpoint_residual<<<kRedBlocks, 256, 0, c->stream>>>(L.n, L.NT, L.U, L.G, L.ld, L.V, L.ld, L.R, L.ld, partial);
        k_sum_partials<<<1, 256, 0, c->stream>>>(kRedBlocks, partial, norm);
        cnt.launches += 2;
        MG_CUDA(cudaGetLastError());
    }

    void sequential_level(int l) {
        Level& L = lv[l];
        for (int64_t t = 1; t <= L.N; ++t)
            phi(l, 1, L.U + (t - 1) * L.n, 1, L.U + t * L.n, 1, L.G + t * L.n, 1, t * L.stride, 0);
    }

    // kind 0: V-cycle, 1: F-cycle (the coarse system solved by an F-cycle and then
    // a V-cycle on the coarse level; one solve when that level is the coarsest)
    void coarse_correction(int l, int kind = 0) {
        Level& F = lv[l];
        Level& C = lv[l + 1];
        // restriction into the coarse mesh's node-major W, g2 (columns = coarse points)
        const Transfer* tr = F.tr;
        k_restrict<<<nblk(C.n * (F.NT + 1)), 256, 0, c->stream>>>(
            C.n, F.NT, F.U, F.ld, F.R, F.ld, tr ? tr->inj.as<int32_t>() : nullptr,
            tr ? tr->PT_ptr.as<int32_t>() : nullptr, tr ? tr->PT_col.as<int32_t>() : nullptr,
            tr ? tr->PT_val.as<double>() : nullptr, tr ? tr->PT_rowsum_inv.as<double>() : nullptr, o.restrict_mode,
            C.W, C.g2, C.ldw);
        cnt.launches += 1;
        MG_CUDA(cudaGetLastError());
        // Phi_c(u2_{c-1}) for all coarse points c = 1..Nc: one batched coarse step
        PhiIO io;
        io.k = (int)C.N;
        io.xprev = C.W;
        io.ld_prev = C.ldw;
        io.guess = C.W + 1;
        io.ld_guess = C.ldw;
        io.xout = C.Vc;
        io.ld_out = C.ldw;
        io.wave = wave;
        io.t0 = C.stride;
        io.tstride = C.stride;
        phi_batch(c, *C.op, io, o.solver, &cnt);
        k_fas_rhs<<<nblk(C.n * (C.N + 1)), 256, 0, c->stream>>>(C.n, C.N, C.W, C.g2, C.Vc, C.ldw, C.gview(), C.view());
        cnt.launches += 1;
        MG_CUDA(cudaGetLastError());
        if (kind == 1 && l + 1 < (int)lv.size() - 1) cycle(l + 1, 1);
        cycle(l + 1, 0);
        k_correct<<<nblk(F.n * F.NT), 256, 0, c->stream>>>(F.n, F.NT, F.U, F.ld, C.view(), C.W, C.ldw,
                                                          tr ? tr->P_ptr.as<int32_t>() : nullptr,
                                                          tr ? tr->P_col.as<int32_t>() : nullptr,
                                                          tr ? tr->P_val.as<double>() : nullptr);
        cnt.launches += 1;
        MG_CUDA(cudaGetLastError());
    }

    void cycle(int l, int kind = 0) {
        if (l == (int)lv.size() - 1) {
            sequential_level(l);
            return;
        }
        relax(l);
        residual(l);
        coarse_correction(l, kind);
        f_relax(l);
    }

    // Nested iterations (Sec. 2.1): the coarsest level's own problem
    // A_L(u) = (R_s a0, 0, ..., 0) solved sequentially, then towards the finest:
    // interpolate to the C-points, F-relax, and one V-cycle below the finest.
    // a0 already sits at point 0 of level 0; the other levels' stores are
    // overwritten.
    void nested_guess(const double* a0) {
        const int L = (int)lv.size();
        const double* keep = wave;
        if (wave_ref) wave = wave_ref;  // the sine reference as the source (Sec. 4.1)
        // a0 on every level's mesh (nodal injection), at point 0 of U and G
        std::vector<const double*> a0l(L, nullptr);
        a0l[0] = a0;
        for (int l = 1; l < L; ++l) {
            Level& P = lv[l - 1];
            Level& C = lv[l];
            const size_t gsz = C.m ? (size_t)C.m * C.n * C.ld : (size_t)(C.N + 1) * C.n;
            MG_CUDA(cudaMemsetAsync(C.G, 0, gsz * sizeof(double), c->stream));
            MG_CUDA(cudaMemsetAsync(C.U, 0, gsz * sizeof(double), c->stream));
            // point 0 of the time-major coarsest store is its first n values; of a slab store, column 0
            double* tmp = C.R ? C.R : C.U + C.n;  // scratch of at least n doubles
            k_gather_state<<<nblk(C.n), 256, 0, c->stream>>>(C.n, P.tr ? P.tr->inj.as<int32_t>() : nullptr,
                                                             a0l[l - 1], tmp);
            if (C.m) {
                k_fill_column<<<nblk(C.n), 256, 0, c->stream>>>(C.n, tmp, C.U, C.ld);
                k_fill_column<<<nblk(C.n), 256, 0, c->stream>>>(C.n, tmp, C.G, C.ld);
            } else {
                MG_CUDA(cudaMemcpyAsync(C.G, tmp, C.n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
                MG_CUDA(cudaMemcpyAsync(C.U, tmp, C.n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            }
            cnt.launches += 3;
            // a contiguous copy of a0 on this mesh for the next gather
            if (!a0stage[l].p || a0stage[l].bytes < C.n * sizeof(double)) a0stage[l].ensure(C.n * sizeof(double));
            MG_CUDA(cudaMemcpyAsync(a0stage[l].p, tmp, C.n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            a0l[l] = a0stage[l].as<double>();
        }
        sequential_level(L - 1);
        for (int l = L - 2; l >= 0; --l) {
            Level& F = lv[l];
            Level& C = lv[l + 1];
            const Transfer* tr = F.tr;
            k_interp_cpoints<<<nblk(F.n * F.NT), 256, 0, c->stream>>>(
                F.n, F.NT, F.view(), F.m, C.view(), tr ? tr->P_ptr.as<int32_t>() : nullptr,
                tr ? tr->P_col.as<int32_t>() : nullptr, tr ? tr->P_val.as<double>() : nullptr);
            cnt.launches += 1;
            MG_CUDA(cudaGetLastError());
            f_relax(l);
            if (l > 0) cycle(l, 0);
        }
        wave = keep;
    }
    DBuf a0stage[8];

    // maximal relative change of the level-0 C-point losses since the last call
    double joule_change(bool first) {
        Level& L = lv[0];
        const MeshLevel& m = c->meshes[L.mesh];
        joule_new.ensure((L.NT + 1) * sizeof(double));
        joule_old.ensure((L.NT + 1) * sizeof(double));
        joule_res.ensure(sizeof(double));
        MG_CUDA(cudaMemsetAsync(joule_new.p, 0, sizeof(double), c->stream));
        k_joule_cpoints<<<(unsigned)L.NT, 256, 0, c->stream>>>(L.n, L.view(), L.m, m.rowptr.as<int32_t>(),
                                                                m.col.as<int32_t>(), m.M.as<double>(), 1.0 / L.dt,
                                                                joule_new.as<double>());
        k_joule_change<<<1, 256, 0, c->stream>>>(L.NT, joule_new.as<double>(), joule_old.as<double>(), first ? 1 : 0,
                                                 joule_res.as<double>());
        cnt.launches += 2;
        MG_CUDA(cudaGetLastError());
        double h = 0.0;
        MG_CUDA(cudaMemcpyAsync(&h, joule_res.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        MG_CUDA(cudaStreamSynchronize(c->stream));
        return h;
    }
    DBuf joule_new, joule_old, joule_res;

    double read_norm() {
        double h = 0.0;
        MG_CUDA(cudaMemcpyAsync(&h, norm, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        MG_CUDA(cudaStreamSynchronize(c->stream));
        return std::sqrt(h);
    }
};

}  // namespace

void check_solver_opts(const mg_solver_opts& so) {
    if (so.max_cg < 1 || so.max_refine < 0 || !(so.cg_tol >= 0.0) || !(so.refine_tol >= 0.0) ||
        !(so.inner_tol >= 0.0) || (so.precision != MG_FP64 && so.precision != MG_FP32_REFINE) || so.cluster < 0 ||
        so.cluster > 16 || !(so.tile == 0 || so.tile == 1 || so.tile == 8 || so.tile == 16 || so.tile == 32) ||
        (so.precond != MG_PRECOND_JACOBI && so.precond != MG_PRECOND_MULTIGRID) || so.smooth < 0 || so.smooth > MG_MAX_NU ||
        !(so.omega >= 0.0 && so.omega < 2.0) || so.path < MG_PATH_AUTO || so.path > MG_PATH_GRAPH ||
        !(so.rows_per_block == 0 || (so.rows_per_block >= 16 && so.rows_per_block <= 4096)) ||
        !(so.coarse_rows_per_block == 0 || (so.coarse_rows_per_block >= 16 && so.coarse_rows_per_block <= 4096)) ||
        !(so.base_tiles == 0 || so.base_tiles == 1 || so.base_tiles == 2 || so.base_tiles == 4) ||
        (so.smoother != MG_SMOOTH_CHEBYSHEV && so.smoother != MG_SMOOTH_JACOBI) ||
        !(so.cheb_ratio == 0.0 || (so.cheb_ratio > 1.0 && so.cheb_ratio <= 1e4)) || so.halo_fusion < 0 ||
        so.halo_fusion > 3 || so.base_cores < 0 || so.base_cores > 2)
        mg_fail(MG_EINVAL, "bad solver options");
}

namespace {

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

void reset_counters(mg_ctx* c) {
    c->counters.ensure(16);
    int64_t init[2] = {0, 0};
    MG_CUDA(cudaMemcpyAsync(c->counters.p, init, 16, cudaMemcpyHostToDevice, c->stream));
}

const char* status_name(int st) {
    switch (st) {
        case MG_ECG_MAXIT: return "MG_ECG_MAXIT";
        case MG_ENEWTON: return "MG_ENEWTON";
        case MG_ETIMEOUT: return "MG_ETIMEOUT";
        case MG_ENONFINITE: return "MG_ENONFINITE";
        default: return "solver failure";
    }
}

void fill_stats(mg_ctx* c, const SolveCounters& cnt, mg_stats* st) {
    unsigned char h[16];
    MG_CUDA(cudaMemcpyAsync(h, c->counters.p, 16, cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(cudaStreamSynchronize(c->stream));
    unsigned long long it;
    int worst;
    std::memcpy(&it, h, 8);
    std::memcpy(&worst, h + 8, 4);
    st->cg_iters = (int64_t)it;
    st->step_solves = cnt.step_solves;
    st->batched_steps = cnt.batched_steps;
    st->launches = cnt.launches;
    st->newton_iters = cnt.newton_iters;
    if (worst < st->worst_status || st->worst_status == 0) st->worst_status = worst;
}

using clk = std::chrono::steady_clock;
double secs(clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); }

mg_status sequential_impl(mg_ctx* c, int level, int64_t N, double T, const double* a0, double* out,
                          const mg_solver_opts* opts, mg_stats* stats) {
    mg_solver_opts so;
    if (opts) so = *opts;
    else mg_solver_defaults(&so);
    check_solver_opts(so);
    if (level < 0 || level >= (int)c->meshes.size() || N <= 0 || !(T > 0.0) || !a0 || !out)
        mg_fail(MG_EINVAL, "mg_sequential: bad arguments");
    auto t0 = clk::now();
    ctx_finalize(c);
    const int64_t n = c->meshes[level].n;
    StepOp& op = ctx_step_op(c, level, T / (double)N);
    const double* wave = ctx_wave_table(c, N, T, 0);
    reset_counters(c);
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        MG_CUDA(cudaStreamSynchronize(c->stream));
    }
    auto t1 = clk::now();
    SolveCounters cnt;
    MG_CUDA(cudaMemcpyAsync(out, a0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    for (int64_t t = 1; t <= N; ++t) {
        PhiIO io;
        io.k = 1;
        io.xprev = out + (t - 1) * n;
        io.ld_prev = 1;
        io.guess = out + (t - 1) * n;  // previous step as the initial guess
        io.ld_guess = 1;
        io.xout = out + t * n;
        io.ld_out = 1;
        io.wave = wave;
        io.t0 = t;
        io.tstride = 0;
        phi_batch(c, op, io, so, &cnt);
    }
    // the per-column statuses are read whether or not the caller wants statistics
    mg_stats local;
    std::memset(&local, 0, sizeof(local));
    mg_stats* st = stats ? stats : &local;
    fill_stats(c, cnt, st);
    st->t_setup = secs(t0, t1);
    st->t_solve = secs(t1, clk::now());
    if (st->worst_status != 0) {
        c->err = "mg_sequential: a step solve did not converge (" + std::string(status_name(st->worst_status)) + ")";
        return (mg_status)st->worst_status;
    }
    return MG_OK;
}

// Sizes of an MGRIT solve's level storage (one pooled allocation, carved in this
// order): per level with a coarsening factor m the iterate U (m slabs of n x ld),
// the FAS right-hand side G (not on level 0), the C-point residual R and the
// values Phi(u) V (n x ld each); the coarsest level U and G time-major; every level
// below the finest also W, g2 and Vc (n x ldw each).
std::vector<size_t> level_storage(const std::vector<Level>& lv) {
    std::vector<size_t> sizes;
    auto plan = [&](int64_t nd) { sizes.push_back((size_t)nd * sizeof(double)); };
    for (int l = 0; l < (int)lv.size(); ++l) {
        const Level& L = lv[l];
        if (L.m) {
            plan(L.m * L.n * L.ld);          // U
            plan(l ? L.m * L.n * L.ld : 0);  // G
            plan(L.n * L.ld);                // R
            plan(L.n * L.ld);                // V
        } else {
            plan((L.N + 1) * L.n);  // U
            plan((L.N + 1) * L.n);  // G
            plan(0);
            plan(0);
        }
        for (int q = 0; q < 3; ++q) plan(l > 0 ? L.n * L.ldw : 0);  // W, g2, Vc
    }
    return sizes;
}

// Device bytes of the graph-path plan of a linear batched step of kpad columns on
// a mesh whose multigrid depths have n[0] (finest) .. n[nd-1] (base) rows: the
// FP32 V-cycle vectors (x on every depth, four K-split copies on the base; s, s',
// y below the base; r below the finest) and the Krylov vectors of the finest depth.
size_t graph_plan_bytes(const std::vector<int64_t>& n, int64_t kpad, int precision) {
    size_t b = 0;
    const int nd = (int)n.size();
    for (int d = 0; d < nd; ++d) {
        const int vecs = (d + 1 == nd ? (nd > 1 ? 4 : 1) : 4) + (d > 0 ? 1 : 0);
        b += (size_t)vecs * kpad * n[d] * sizeof(float);
    }
    b += (size_t)kpad * n[0] * (precision == MG_FP64 ? 4 * 8 + 4 : 2 * 8 + 4 * 4);
    return b;
}

// Estimated device bytes an MGRIT solve of N steps with options o allocates in the
// context: the level storage (exact) and the step plans of its relaxation batches
// (one per level and batch width; Newton plans add the per-column Jacobians, their
// FP32 copies and scaled values on every depth and the banded base factor).
size_t mgrit_work_estimate(mg_ctx* c, int64_t N, const mg_opts& o) {
    if (N <= 0 || o.levels < 1 || o.levels > 8) mg_fail(MG_EINVAL, "bad solve arguments");
    for (int l = 0; l < o.levels; ++l)
        if (o.space_level[l] < 0 || o.space_level[l] >= (int)c->meshes.size()) mg_fail(MG_EINVAL, "bad space level");
    std::vector<Level> lv(o.levels);
    int64_t stride = 1;
    for (int l = 0; l < o.levels; ++l) {
        Level& L = lv[l];
        L.mesh = o.space_level[l];
        L.n = c->meshes[L.mesh].n;
        L.N = N / stride;
        if (l < o.levels - 1 && o.levels > 1) {
            L.m = std::max(1, o.m[l]);
            L.NT = L.N / L.m;
            L.ld = round_up(L.NT + 1, 4);
            stride *= L.m;
        }
        if (l > 0) L.ldw = round_up(L.N + 1, 4);
    }
    size_t bytes = 0;
    if (o.levels > 1)
        for (auto s : level_storage(lv)) bytes += s;
    // one batched-step plan per (mesh, batch width) the solve relaxes with
    std::set<std::pair<int, int64_t>> shapes;
    for (int l = 0; l < o.levels; ++l) {
        const int64_t k = o.levels > 1 && l < o.levels - 1 ? lv[l].NT : 1;
        shapes.insert({lv[l].mesh, (k + 15) / 16 * 16});
    }
    for (const auto& sh : shapes) {
        if (sh.second < MG_GRAPH_MIN_COLUMNS) continue;  // cluster path: small shared work vectors
        std::vector<int64_t> n;
        std::vector<int> bw;
        for (int m = sh.first; m >= 0; m = c->meshes[m].parent_mesh) {
            n.push_back(c->meshes[m].n);
            bw.push_back(c->meshes[m].ell_bw);
            if (o.solver.precond != MG_PRECOND_MULTIGRID) break;
        }
        bytes += graph_plan_bytes(n, sh.second, o.solver.precision);
        if (mesh_is_nonlinear(c, sh.first)) {
            int64_t rows = 0;
            for (auto x : n) rows += x;
            const int W = c->meshes[sh.first].ell_W;
            bytes += (size_t)sh.second * rows * (W * (8 + 4 + 4) + 16);
            bytes += (size_t)sh.second * n.back() * (2 * bw.back() + 1) * sizeof(float) * 2;
        }
    }
    return bytes;
}

mg_status solve_impl(mg_ctx* c, int64_t N, double T, const double* a0, double* out, const mg_opts* opts,
                     mg_stats* stats) {
    mg_opts o;
    if (opts) o = *opts;
    else mg_opts_defaults(&o);
    check_solver_opts(o.solver);
    if (N <= 0 || !(T > 0.0) || !a0 || !out || o.levels < 1 || o.levels > 8 || o.relax < 0 || o.relax > 4 ||
        o.max_iter < 0 || !(o.tol >= 0.0) || o.restrict_mode < 0 || o.restrict_mode > 2 || o.cycle < 0 ||
        o.cycle > 1 || o.nested < 0 || o.nested > 2 || o.stop_rule < 0 || o.stop_rule > 1 ||
        !(o.step_tol_ratio >= 0.0))
        mg_fail(MG_EINVAL, "mg_solve: bad arguments");
    auto t0 = clk::now();
    ctx_finalize(c);
    for (int l = 0; l < o.levels; ++l)
        if (o.space_level[l] < 0 || o.space_level[l] >= (int)c->meshes.size())
            mg_fail(MG_EINVAL, "mg_solve: bad space level");
    if (o.levels == 1) {
        mg_solver_opts so = o.solver;
        mg_status st = sequential_impl(c, o.space_level[0], N, T, a0, out, &so, stats);
        if (stats) stats->iters = 0;
        return st;
    }
    Solver S{c, N, T, o};
    S.lv.resize(o.levels);
    int64_t stride = 1;
    for (int l = 0; l < o.levels; ++l) {
        Level& L = S.lv[l];
        L.mesh = o.space_level[l];
        L.n = c->meshes[L.mesh].n;
        if (N % stride) mg_fail(MG_EINVAL, "N must be divisible by the product of the coarsening factors");
        L.N = N / stride;
        L.stride = stride;
        L.dt = T / (double)L.N;
        L.op = &ctx_step_op(c, L.mesh, L.dt);
        if (l < o.levels - 1) {
            L.m = o.m[l];
            if (L.m < 1 || L.N % L.m) mg_fail(MG_EINVAL, "N must be divisible by the product of the coarsening factors");
            L.NT = L.N / L.m;
            L.ld = round_up(L.NT + 1, 4);
            int cm = o.space_level[l + 1];
            if (cm != L.mesh) {
                if (c->meshes[cm].n > L.n) mg_fail(MG_EINVAL, "coarse space level must not be finer");
                L.tr = &ctx_transfer(c, L.mesh, cm);
            }
            stride *= L.m;
        } else {
            L.m = 0;
            L.NT = L.N;
            L.ld = 0;
        }
    }
    // storage
    for (int l = 1; l < o.levels; ++l) S.lv[l].ldw = round_up(S.lv[l].N + 1, 4);
    std::vector<size_t> sizes = level_storage(S.lv);
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t bytes = 0;
    for (auto s : sizes) bytes += r256(s);
    bytes += r256(S.kRedBlocks * sizeof(double)) + r256(sizeof(double));
    // one pooled allocation, carved per level
    c->solve_buf[0].ensure(bytes);
    char* p = (char*)c->solve_buf[0].p;
    auto take = [&](size_t b) -> double* {
        double* r = b ? (double*)p : nullptr;
        p += (b + 255) / 256 * 256;
        return r;
    };
    size_t q = 0;
    for (int l = 0; l < o.levels; ++l) {
        Level& L = S.lv[l];
        L.U = take(sizes[q++]);
        L.G = take(sizes[q++]);
        L.R = take(sizes[q++]);
        L.V = take(sizes[q++]);
        L.W = take(sizes[q++]);
        L.g2 = take(sizes[q++]);
        L.Vc = take(sizes[q++]);
    }
    S.partial = take(S.kRedBlocks * sizeof(double));
    S.norm = take(sizeof(double));
    S.wave = ctx_wave_table(c, N, T, 0);
    if (o.nested == 2) S.wave_ref = ctx_wave_table(c, N, T, 1);
    reset_counters(c);
    Level& L0 = S.lv[0];
    MG_CUDA(cudaMemsetAsync(L0.U, 0, L0.m * L0.n * L0.ld * sizeof(double), c->stream));
    k_fill_column<<<nblk(L0.n), 256, 0, c->stream>>>(L0.n, a0, L0.U, L0.ld);
    S.cnt.launches += 1;
    MG_CUDA(cudaGetLastError());
    if (o.nested) S.nested_guess(a0);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    MG_CUDA(cudaStreamSynchronize(c->stream));
    auto t1 = clk::now();
    std::vector<double> hist;
    double r0 = 0.0;
    int it = 0;
    bool converged = false;
    // inexact step solves: tolerance proportional to the current relative residual
    const bool adaptive = o.step_tol_ratio > 0.0 && o.stop_rule == 0;
    const double tol_cg = o.solver.cg_tol, tol_ref = o.solver.refine_tol, tol_newton = o.solver.newton_tol;
    auto set_step_tol = [&](double rho) {
        if (!adaptive) return;
        S.o.solver.cg_tol = std::max(tol_cg, o.step_tol_ratio * rho);
        S.o.solver.refine_tol = std::max(tol_ref, o.step_tol_ratio * rho);
        // Newton steps: the relative update at which Newton stops
        S.o.solver.newton_tol = std::max(tol_newton, o.step_tol_ratio * rho);
    };
    set_step_tol(1.0);
    // stagnation (residual rule only): for kStallIters iterations in a row no residual
    // below kStallDrop times the best one so far (slow but steady convergence, e.g.
    // 0.95 per iteration, keeps making such progress; a residual that only wanders at
    // a floor does not)
    constexpr int kStallIters = 5;
    constexpr double kStallDrop = 0.9;
    double best = INFINITY;
    int since_best = 0;
    bool stalled = false;
    double ref = 1.0;
    for (it = 0;; ++it) {
        S.relax(0);
        S.residual(0);
        double rn = o.stop_rule == 1 ? S.joule_change(it == 0) : S.read_norm();
        hist.push_back(rn);
        if (mg_trace_level() >= 1)
            std::fprintf(stderr, "[mgrit] iteration %d  residual %.4e  %.3f s  step-solves %lld  newton %lld\n", it,
                         rn, secs(t1, clk::now()), (long long)S.cnt.step_solves, (long long)S.cnt.newton_iters);
        if (it == 0) r0 = rn;
        ref = (o.tol_relative && o.stop_rule == 0) ? r0 : 1.0;
        if (rn <= o.tol * ref) {
            converged = true;
            break;
        }
        if (rn != rn || it >= o.max_iter) break;
        if (o.stop_rule == 0) {
            if (rn < kStallDrop * best || it == 0) {
                best = std::min(best, rn);
                since_best = 0;
            } else if (++since_best >= kStallIters) {
                stalled = true;
                break;
            }
        }
        set_step_tol(r0 > 0.0 ? rn / r0 : 1.0);
        S.coarse_correction(0, o.cycle);
    }
    k_to_time_major<<<nblk(L0.n * (N + 1)), 256, 0, c->stream>>>(L0.n, N, L0.view(), out);
    S.cnt.launches += 1;
    MG_CUDA(cudaGetLastError());
    // the per-column statuses are read whether or not the caller wants statistics
    mg_stats local;
    std::memset(&local, 0, sizeof(local));
    mg_stats* st = stats ? stats : &local;
    fill_stats(c, S.cnt, st);
    st->iters = it;
    st->n_hist = (int)std::min<size_t>(hist.size(), 64);
    for (int k = 0; k < st->n_hist; ++k) st->res_hist[k] = hist[k];
    st->t_setup = secs(t0, t1);
    st->t_solve = secs(t1, clk::now());
    if (st->worst_status != 0) {
        c->err = "mg_solve: a step solve did not converge (" + std::string(status_name(st->worst_status)) + ")";
        return (mg_status)st->worst_status;
    }
    if (converged) return MG_OK;
    char msg[256];
    const double last = hist.empty() ? 0.0 : hist.back();
    std::snprintf(msg, sizeof msg, "mg_solve: %s after %d iterations: %s %.3e (%.3e of the first), tolerance %.3e",
                  stalled ? "residual stagnated" : (last != last ? "residual is not finite" : "max_iter reached"), it,
                  o.stop_rule == 1 ? "Joule-loss change" : "residual", last, r0 > 0.0 ? last / r0 : 0.0,
                  o.tol * ref);
    c->err = msg;
    return stalled ? MG_ESTALLED : MG_EMGRIT_MAXIT;
}

}  // namespace

// A few MGRIT iterations with the given options from a0 = 0 (library-owned
// trajectory buffer), for the coarsening planner: the residual history and the
// seconds the iterations took (set-up excluded).
void mgrit_probe(mg_ctx* c, int64_t N, double T, const mg_opts& opts, int iters, std::vector<double>& hist,
                 double& seconds) {
    mg_opts o = opts;
    o.max_iter = iters;
    o.tol = 0.0;
    o.tol_relative = 0;
    const int64_t n = c->meshes[o.space_level[0]].n;
    c->host_in.ensure(n * sizeof(double));
    c->host_out.ensure((size_t)(N + 1) * n * sizeof(double));
    MG_CUDA(cudaMemsetAsync(c->host_in.p, 0, n * sizeof(double), c->stream));
    mg_stats st;
    const mg_status rc = solve_impl(c, N, T, c->host_in.as<double>(), c->host_out.as<double>(), &o, &st);
    if (rc != MG_OK && rc != MG_EMGRIT_MAXIT && rc != MG_ESTALLED) mg_fail(rc, "mgrit_probe: " + c->err);
    c->err.clear();
    hist.assign(st.res_hist, st.res_hist + st.n_hist);
    seconds = st.t_solve;
}

extern mg_status mg_guarded_call(mg_ctx* c, void (*fn)(void*), void* arg);

template <class F>
static mg_status run(mg_ctx* c, F&& f) {
    mg_status out = MG_OK;
    struct Box {
        F* f;
        mg_status* out;
    } box{&f, &out};
    mg_status st = mg_guarded_call(
        c, [](void* a) { auto* b = (Box*)a; *b->out = (*b->f)(); }, &box);
    return st != MG_OK ? st : out;
}

extern "C" {

void mg_solver_defaults(mg_solver_opts* s) {
    if (!s) return;
    std::memset(s, 0, sizeof(*s));
    s->cg_tol = 1e-13;
    s->refine_tol = 1e-13;
    s->inner_tol = 3e-2;
    s->max_cg = 2000;
    s->max_refine = 30;
    s->precision = MG_FP64;
    s->cluster = 0;
    s->tile = 0;
    s->precond = MG_PRECOND_MULTIGRID;
    s->smooth = 5;
    s->omega = 0.7;
    s->newton_tol = 1e-8;
    s->max_newton = 100;
    s->max_halvings = 40;
    s->newton_lin_tol = 1e-6;
    s->smoother = MG_SMOOTH_CHEBYSHEV;
    s->cheb_ratio = 30.0;
}

mg_status mg_smoother_weights(const mg_solver_opts* so, double lam, int nu, float* w) {
    if (!so || !w || nu < 1 || nu > MG_MAX_NU || !(lam >= 0.0) ||
        (so->smoother != MG_SMOOTH_CHEBYSHEV && so->smoother != MG_SMOOTH_JACOBI) ||
        !(so->cheb_ratio == 0.0 || (so->cheb_ratio > 1.0 && so->cheb_ratio <= 1e4)) ||
        !(so->omega >= 0.0 && so->omega < 2.0))
        return MG_EINVAL;
    smoother_weights(lam, *so, nu, w);
    return MG_OK;
}

void mg_opts_defaults(mg_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->levels = 2;
    for (int l = 0; l < 8; ++l) o->m[l] = 16;
    o->relax = 1;
    o->tol = 1e-10;
    o->tol_relative = 1;
    o->max_iter = 50;
    o->restrict_mode = 2;
    mg_solver_defaults(&o->solver);
}

mg_status mg_step(mg_ctx* c, int level, int64_t N, double T, int64_t dt_mult, int k, int64_t i0, int64_t istride,
                  const double* x_in, int64_t ld_in, double* x_out, int64_t ld_out, int guess,
                  const mg_solver_opts* opts, mg_stats* stats) {
    return run(c, [&]() -> mg_status {
        mg_solver_opts so;
        if (opts) so = *opts;
        else mg_solver_defaults(&so);
        check_solver_opts(so);
        if (level < 0 || level >= (int)c->meshes.size() || N <= 0 || !(T > 0.0) || dt_mult <= 0 || k <= 0 ||
            !x_in || !x_out || ld_in < k || ld_out < k || i0 < 0 || i0 > N || istride < 0 ||
            i0 + (int64_t)(k - 1) * istride > N)
            mg_fail(MG_EINVAL, "mg_step: bad arguments");
        ctx_finalize(c);
        StepOp& op = ctx_step_op(c, level, (double)dt_mult * T / (double)N);
        const double* wave = ctx_wave_table(c, N, T, 0);
        reset_counters(c);
        auto t1 = clk::now();
        PhiIO io;
        io.k = k;
        io.xprev = x_in;
        io.ld_prev = ld_in;
        io.guess = guess ? x_out : nullptr;
        io.ld_guess = ld_out;
        io.xout = x_out;
        io.ld_out = ld_out;
        io.wave = wave;
        io.t0 = i0;
        io.tstride = istride;
        SolveCounters cnt;
        phi_batch(c, op, io, so, &cnt);
        if (stats) {
            std::memset(stats, 0, sizeof(*stats));
            fill_stats(c, cnt, stats);
            stats->t_solve = secs(t1, clk::now());
            if (stats->worst_status != 0) return (mg_status)stats->worst_status;
        }
        return MG_OK;
    });
}

mg_status mg_joule_losses(mg_ctx* c, int level, int64_t N, double T, const double* traj, double* losses) {
    return run(c, [&]() -> mg_status {
        if (level < 0 || level >= (int)c->meshes.size() || N <= 0 || !(T > 0.0) || !traj || !losses)
            mg_fail(MG_EINVAL, "mg_joule_losses: bad arguments");
        ctx_finalize(c);
        const MeshLevel& m = c->meshes[level];
        MG_CUDA(cudaMemsetAsync(losses, 0, sizeof(double), c->stream));
        LevelView v{const_cast<double*>(traj), m.n, 0, 0, 0};
        k_joule_traj<<<(unsigned)N, 256, 0, c->stream>>>(m.n, v, m.rowptr.as<int32_t>(), m.col.as<int32_t>(),
                                                          m.M.as<double>(), (double)N / T, losses);
        MG_CUDA(cudaGetLastError());
        return MG_OK;
    });
}

mg_status mg_sequential(mg_ctx* c, int level, int64_t N, double T, const double* a0, double* out,
                        const mg_solver_opts* opts, mg_stats* stats) {
    return run(c, [&]() { return sequential_impl(c, level, N, T, a0, out, opts, stats); });
}

mg_status mg_solve(mg_ctx* c, int64_t N, double T, const double* a0, double* out, const mg_opts* opts,
                   mg_stats* stats) {
    return run(c, [&]() { return solve_impl(c, N, T, a0, out, opts, stats); });
}

mg_status mg_solve_work_bytes(mg_ctx* c, int64_t N, const mg_opts* opts, int64_t* bytes) {
    return run(c, [&]() -> mg_status {
        if (!bytes) mg_fail(MG_EINVAL, "mg_solve_work_bytes: bad arguments");
        mg_opts o;
        if (opts) o = *opts;
        else mg_opts_defaults(&o);
        *bytes = (int64_t)mgrit_work_estimate(c, N, o);
        return MG_OK;
    });
}

mg_status mg_release_work(mg_ctx* c) {
    return run(c, [&]() -> mg_status {
        MG_CUDA(cudaStreamSynchronize(c->stream));
        ctx_drop_plans(c);
        for (auto& b : c->solve_buf) b.release();
        for (auto& b : c->ws) b.release();
        c->host_in.release();
        c->host_out.release();
        return MG_OK;
    });
}

mg_status mg_solve_host(mg_ctx* c, int64_t N, double T, const double* a0_host, double* out_host, const mg_opts* opts,
                        mg_stats* stats) {
    return run(c, [&]() -> mg_status {
        if (!a0_host || !out_host || N <= 0) mg_fail(MG_EINVAL, "mg_solve_host: bad arguments");
        mg_opts o;
        if (opts) o = *opts;
        else mg_opts_defaults(&o);
        if (o.space_level[0] < 0 || o.space_level[0] >= (int)c->meshes.size())
            mg_fail(MG_EINVAL, "mg_solve_host: bad space level");
        const int64_t n = c->meshes[o.space_level[0]].n;
        c->host_in.ensure(n * sizeof(double));
        c->host_out.ensure((size_t)(N + 1) * n * sizeof(double));
        MG_CUDA(cudaMemcpyAsync(c->host_in.p, a0_host, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        mg_status st = solve_impl(c, N, T, c->host_in.as<double>(), c->host_out.as<double>(), &o, stats);
        MG_CUDA(cudaMemcpyAsync(out_host, c->host_out.p, (size_t)(N + 1) * n * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
        MG_CUDA(cudaStreamSynchronize(c->stream));
        return st;
    });
}

mg_status mg_sequential_host(mg_ctx* c, int level, int64_t N, double T, const double* a0_host, double* out_host,
                             const mg_solver_opts* opts, mg_stats* stats) {
    return run(c, [&]() -> mg_status {
        if (!a0_host || !out_host || N <= 0 || level < 0 || level >= (int)c->meshes.size())
            mg_fail(MG_EINVAL, "mg_sequential_host: bad arguments");
        const int64_t n = c->meshes[level].n;
        c->host_in.ensure(n * sizeof(double));
        c->host_out.ensure((size_t)(N + 1) * n * sizeof(double));
        MG_CUDA(cudaMemcpyAsync(c->host_in.p, a0_host, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        mg_status st = sequential_impl(c, level, N, T, c->host_in.as<double>(), c->host_out.as<double>(), opts, stats);
        MG_CUDA(cudaMemcpyAsync(out_host, c->host_out.p, (size_t)(N + 1) * n * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
        MG_CUDA(cudaStreamSynchronize(c->stream));
        return st;
    });
}

}  // extern "C"
