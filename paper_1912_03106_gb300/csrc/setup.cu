// Context, mesh set-up and P1 assembly of libmgrit_em.so.
//
// Assembly (Sec. 3.1, Eq. semi_discrete_system): per triangle T with area |T|
// and barycentric gradients G (3 x 2), K_T = nu |T| G G^T, M_T = sigma |T|/12
// (1 + delta_ab), and the phase loads F_s = sign * |T|/3 per vertex.  The CSR
// pattern of the interior unknowns is built on the host; element values are
// computed on the device and summed into CSR slots by a gather over a
// precomputed slot -> (element, a, b) list, so the sums have a fixed order and
// repeated runs are bitwise identical.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>

#include "internal.h"

#include <cooperative_groups.h>
namespace cg = cooperative_groups;

// ------------------------------------------------------------------ errors

[[noreturn]] void mg_fail(mg_status st, const std::string& msg) { throw MgError{st, msg}; }

void mg_check_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        mg_status st = (e == cudaErrorMemoryAllocation) ? MG_ENOMEM : MG_ECUDA;
        mg_fail(st, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void DBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

void DBuf::ensure(size_t nbytes) {
    if (nbytes <= bytes && p) return;
    release();
    if (nbytes == 0) nbytes = 16;
    MG_CUDA(cudaMalloc(&p, nbytes));
    bytes = nbytes;
}

int mg_trace_level() {
    static const int level = [] {
        const char* v = std::getenv("MGRIT_EM_TRACE");
        return v ? std::atoi(v) : 0;
    }();
    return level;
}

void ctx_drop_plans(mg_ctx* c) {
    for (auto* p : c->nplans) newton_plan_delete(p);
    c->nplans.clear();
    for (auto* p : c->plans) graph_plan_delete(p);
    c->plans.clear();
}

mg_ctx::~mg_ctx() {
    ctx_drop_plans(this);
    for (auto& q : nl) nl_mesh_delete(q.second);
    for (auto* o : ops) delete o;
    for (auto& t : transfers) delete t.second;
}

template <class F>
static mg_status guarded(mg_ctx* c, F&& f) {
    if (!c) return MG_EINVAL;
    try {
        c->err.clear();
        MG_CUDA(cudaSetDevice(c->device));
        f();
        return MG_OK;
    } catch (const MgError& e) {
        c->err = e.msg;
        return e.st;
    } catch (const std::bad_alloc&) {
        c->err = "host allocation failed";
        return MG_ENOMEM;
    } catch (...) {
        c->err = "unexpected internal error";
        return MG_ECUDA;
    }
}

// ------------------------------------------------------------------ kernels

__global__ void k_elem_geometry(int64_t n_tri, const int32_t* __restrict__ tri, const double* __restrict__ xy,
                                double* __restrict__ area, double* __restrict__ grad, int* __restrict__ flag) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_tri) return;
    double px[3], py[3];
    for (int a = 0; a < 3; ++a) {
        int v = tri[3 * e + a];
        px[a] = xy[2 * v];
        py[a] = xy[2 * v + 1];
    }
    double det = (px[1] - px[0]) * (py[2] - py[0]) - (py[1] - py[0]) * (px[2] - px[0]);
    if (!(det > 0.0)) {
        atomicExch(flag, 1);
        det = 1.0;
    }
    area[e] = 0.5 * det;
    // gradient of the barycentric coordinate of vertex a: the opposite edge turned
    // by -90 degrees, divided by 2|T|
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, d = (a + 2) % 3;
        grad[6 * e + 2 * a] = (py[b] - py[d]) / det;
        grad[6 * e + 2 * a + 1] = (px[d] - px[b]) / det;
    }
}

__global__ void k_elem_linear(int64_t n_tri, const double* __restrict__ area, const double* __restrict__ grad,
                              const double* __restrict__ sigma, const double* __restrict__ nu,
                              double* __restrict__ elemK, double* __restrict__ elemM) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_tri) return;
    const double A = area[e];
    const double* g = grad + 6 * e;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double gg = g[2 * a] * g[2 * b] + g[2 * a + 1] * g[2 * b + 1];
            elemK[9 * e + 3 * a + b] = nu[e] * A * gg;
            elemM[9 * e + 3 * a + b] = sigma[e] * A * (a == b ? 2.0 : 1.0) / 12.0;
        }
}

// CSR slot s = sum of its element contributions, in list order.
__global__ void k_gather_slots(int64_t nnz, const int32_t* __restrict__ ptr, const int32_t* __restrict__ src,
                               const double* __restrict__ elem, double* __restrict__ out) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    double acc = 0.0;
    for (int32_t q = ptr[s]; q < ptr[s + 1]; ++q) acc += elem[src[q]];
    out[s] = acc;
}

// F[phase * n + i] = sum over incident source elements of sign * |T| / 3.
__global__ void k_phase_loads(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ src,
                              const int32_t* __restrict__ elem_src, const double* __restrict__ area,
                              double* __restrict__ F) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int32_t q = ptr[i]; q < ptr[i + 1]; ++q) {
        int e = src[q] / 3;
        int s = elem_src[e];
        if (s < 0) continue;
        double v = area[e] / 3.0;
        acc[s >> 1] += (s & 1) ? -v : v;
    }
    for (int p = 0; p < 3; ++p) F[p * n + i] = acc[p];
}

// ELL values of L = M/dt + K (and M) from the CSR values; padding entries are 0.
__global__ void k_ell_values(int64_t nW, const int32_t* __restrict__ slot, const double* __restrict__ K,
                             const double* __restrict__ M, double inv_dt, double* __restrict__ L64,
                             double* __restrict__ M64, float* __restrict__ L32, float* __restrict__ Llo32,
                             float* __restrict__ M32, float* __restrict__ Mlo32) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nW) return;
    int32_t s = slot[q];
    double l = 0.0, m = 0.0;
    if (s >= 0) {
        m = M[s];
        l = m * inv_dt + K[s];
    }
    L64[q] = l;
    M64[q] = m;
    const float hi = (float)l;
    L32[q] = hi;
    Llo32[q] = (float)(l - (double)hi);  // exact difference, rounded once
    const float mh = (float)m;
    M32[q] = mh;
    Mlo32[q] = (float)(m - (double)mh);
}

__global__ void k_ell_diag(int64_t n, int W, const int32_t* __restrict__ col, const double* __restrict__ L64,
                           double* __restrict__ dinv64, float* __restrict__ dinv32, int* __restrict__ flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int w = 0; w < W; ++w)
        if (col[w * n + i] == i) d += L64[w * n + i];
    if (!(d > 0.0)) {
        atomicExch(flag, 1);
        d = 1.0;
    }
    dinv64[i] = 1.0 / d;
    dinv32[i] = (float)(1.0 / d);
}

__global__ void k_ell_scaled(int64_t nW, int64_t n, const int32_t* __restrict__ col, const double* __restrict__ L64,
                             const double* __restrict__ dinv64, float* __restrict__ LD32) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nW) return;
    LD32[q] = (float)(L64[q] * dinv64[col[q]]);
}

// Gershgorin bound of the spectrum of D^-1 L: max over rows of sum_j |L_ij| / L_ii,
// rounded up to float; a positive float's bits order like the value, so the
// maximum is an unsigned atomicMax.
__global__ void k_ell_gershgorin(int64_t n, int W, const double* __restrict__ L64, const double* __restrict__ dinv64,
                                 unsigned* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = 0.0;
    for (int w = 0; w < W; ++w) a += fabs(L64[w * n + i]);
    atomicMax(out, __float_as_uint(__double2float_ru(a * dinv64[i])));
}

// Dense [A | I] (n x 2n, row-major) of the base operator for Gauss-Jordan inversion.
__global__ void k_dense_aug(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double* __restrict__ K, const double* __restrict__ M, double inv_dt,
                            double* __restrict__ aug) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t s = rowptr[i]; s < rowptr[i + 1]; ++s) aug[i * 2 * n + col[s]] = M[s] * inv_dt + K[s];
    aug[i * 2 * n + n + i] = 1.0;
}

// Whole Gauss-Jordan sweep on [A | I] in one cooperative launch.  Pivot k
// needs column k and row k as they stood after pivot k-1; the threads that
// produce those entries also copy them into ping-pong buffers, so one grid
// barrier per pivot suffices.  Only columns k..n+k change at pivot k: the
// columns left of k are already unit vectors and those right of n+k are still
// untouched identity columns.  Every block reads the same pivot after the
// barrier, so a non-positive pivot ends all blocks together.
__global__ void k_gj_sweep(int64_t n, double* __restrict__ aug, double* __restrict__ colbuf,
                           double* __restrict__ rowbuf, int* __restrict__ flag) {
    cg::grid_group grid = cg::this_grid();
    const int64_t W = 2 * n;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = tid; q < n; q += nth) colbuf[q] = aug[q * W];
    for (int64_t q = tid; q < W; q += nth) rowbuf[q] = aug[q];
    grid.sync();
    for (int64_t k = 0; k < n; ++k) {
        const double* ck = colbuf + (k & 1) * n;
        const double* rk = rowbuf + (k & 1) * W;
        double* cn = colbuf + ((k + 1) & 1) * n;
        double* rn = rowbuf + ((k + 1) & 1) * W;
        const double piv = rk[k];
        if (!(piv > 0.0)) {
            if (tid == 0) atomicExch(flag, 1);
            return;
        }
        if (tid == 0 && k + 1 < n) rn[n + k + 1] = aug[(k + 1) * W + n + k + 1];
        for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
            const double f = ck[i];
            double* row = aug + i * W;
            for (int64_t j = k + threadIdx.x; j <= n + k; j += blockDim.x) {
                const double pk = rk[j] / piv;
                const double v = (i == k) ? pk : row[j] - f * pk;
                row[j] = v;
                if (j == k + 1) cn[i] = v;
                if (i == k + 1) rn[j] = v;
            }
        }
        grid.sync();
    }
}

__global__ void k_gj_extract(int64_t n, const double* __restrict__ aug, float* __restrict__ inv) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n * n) return;
    int64_t i = q / n, j = q % n;
    inv[q] = (float)aug[i * 2 * n + n + j];
}

// PWM switching functions of Sec. 3.2-3.3 on t_i = i * (T / N).
__global__ void k_pwm_table(int64_t N, double T_over_N, double w, double mod_index, int carrier,
                            int64_t q_int, double f_c, double phi1, double phi2, int8_t* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > N) return;
    double t = __dmul_rn((double)i, T_over_N);
    double ph;
    if (q_int >= 0) {
        ph = (double)((q_int * i) % N) / (double)N;  // exact carrier phase from integers
    } else {
        double x = __dmul_rn(f_c, t);
        ph = x - floor(x);
    }
    double c = carrier == 0 ? 2.0 * ph - 1.0 : 1.0 - 4.0 * fabs(ph - 0.5);
    const double phis[3] = {0.0, phi1, phi2};
    for (int s = 0; s < 3; ++s) {
        double r = mod_index * sin(__dadd_rn(__dmul_rn(w, t), phis[s]));
        double d = r - c;
        out[3 * i + s] = (int8_t)((d > 0.0) - (d < 0.0));
    }
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Start-up factor of Sec. 3.3: 0.5 (1 - cos(pi t / t_ramp)) for t < t_ramp, else 1.
__device__ __forceinline__ double ramp_factor(double t, double t_ramp) {
    return (t_ramp > 0.0 && t < t_ramp) ? 0.5 * (1.0 - cos(M_PI * t / t_ramp)) : 1.0;
}

// Source waveform w_s(t_i) = alpha(t_i) b_s(t_i) from the PWM sign table.
__global__ void k_wave_pwm(int64_t N, double T_over_N, double t_ramp, const int8_t* __restrict__ signs,
                           double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > N) return;
    const double a = ramp_factor(__dmul_rn((double)i, T_over_N), t_ramp);
    for (int s = 0; s < 3; ++s) out[3 * i + s] = a * (double)signs[3 * i + s];
}

// w_s(t_i) = alpha(t_i) r_s(t_i): the sine reference of Eq. machine_reference_signal.
__global__ void k_wave_reference(int64_t N, double T_over_N, double w, double mod_index, double phi1, double phi2,
                                 double t_ramp, double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > N) return;
    const double t = __dmul_rn((double)i, T_over_N);
    const double a = ramp_factor(t, t_ramp);
    const double phis[3] = {0.0, phi1, phi2};
    for (int s = 0; s < 3; ++s) out[3 * i + s] = a * (mod_index * sin(__dadd_rn(__dmul_rn(w, t), phis[s])));
}

// ------------------------------------------------------------------ assembly

static int read_flag(mg_ctx* c) {
    int h = 0;
    MG_CUDA(cudaMemcpyAsync(&h, c->flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(cudaStreamSynchronize(c->stream));
    return h;
}

static void clear_flag(mg_ctx* c) {
    c->flag.ensure(sizeof(int) * 4);
    MG_CUDA(cudaMemsetAsync(c->flag.p, 0, sizeof(int) * 4, c->stream));
}

static void build_pattern(MeshLevel& m) {
    const int64_t nt = m.n_tri;
    std::vector<std::vector<int32_t>> rows(m.n);
    for (int64_t e = 0; e < nt; ++e)
        for (int a = 0; a < 3; ++a) {
            int32_t da = m.node2dof[m.tri[3 * e + a]];
            if (da < 0) continue;
            for (int b = 0; b < 3; ++b) {
                int32_t db = m.node2dof[m.tri[3 * e + b]];
                if (db >= 0) rows[da].push_back(db);
            }
        }
    m.rowptr_h.assign(m.n + 1, 0);
    m.col_h.clear();
    for (int64_t i = 0; i < m.n; ++i) {
        auto& r = rows[i];
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
        m.col_h.insert(m.col_h.end(), r.begin(), r.end());
        m.rowptr_h[i + 1] = (int32_t)m.col_h.size();
    }
    m.nnz = (int64_t)m.col_h.size();
    if (m.nnz >= (int64_t)INT32_MAX) mg_fail(MG_EINVAL, "mesh too large for int32 CSR indices");
    m.diag_h.assign(m.n, -1);
    auto slot_of = [&](int32_t r, int32_t cidx) -> int32_t {
        auto b = m.col_h.begin() + m.rowptr_h[r];
        auto e = m.col_h.begin() + m.rowptr_h[r + 1];
        auto it = std::lower_bound(b, e, cidx);
        return (int32_t)(it - m.col_h.begin());
    };
    for (int64_t i = 0; i < m.n; ++i) m.diag_h[i] = slot_of((int32_t)i, (int32_t)i);
    // slot -> element contributions (counting sort keeps element order inside a slot)
    std::vector<int32_t> cnt(m.nnz + 1, 0), slot_of_src(9 * nt, -1);
    for (int64_t e = 0; e < nt; ++e)
        for (int a = 0; a < 3; ++a) {
            int32_t da = m.node2dof[m.tri[3 * e + a]];
            if (da < 0) continue;
            for (int b = 0; b < 3; ++b) {
                int32_t db = m.node2dof[m.tri[3 * e + b]];
                if (db < 0) continue;
                int32_t s = slot_of(da, db);
                slot_of_src[9 * e + 3 * a + b] = s;
                cnt[s + 1]++;
            }
        }
    std::partial_sum(cnt.begin(), cnt.end(), cnt.begin());
    std::vector<int32_t> src(cnt[m.nnz]), fill(cnt.begin(), cnt.end() - 1);
    for (int64_t q = 0; q < 9 * nt; ++q)
        if (slot_of_src[q] >= 0) src[fill[slot_of_src[q]]++] = (int32_t)q;
    upload(m.slot_ptr, cnt);
    upload(m.slot_src, src);
    // dof -> incident (element, vertex) pairs for the load vectors
    std::vector<int32_t> lc(m.n + 1, 0);
    for (int64_t e = 0; e < nt; ++e)
        for (int a = 0; a < 3; ++a) {
            int32_t d = m.node2dof[m.tri[3 * e + a]];
            if (d >= 0) lc[d + 1]++;
        }
    std::partial_sum(lc.begin(), lc.end(), lc.begin());
    std::vector<int32_t> lsrc(lc[m.n]), lfill(lc.begin(), lc.end() - 1);
    for (int64_t e = 0; e < nt; ++e)
        for (int a = 0; a < 3; ++a) {
            int32_t d = m.node2dof[m.tri[3 * e + a]];
            if (d >= 0) lsrc[lfill[d]++] = (int32_t)(3 * e + a);
        }
    upload(m.load_ptr, lc);
    upload(m.load_src, lsrc);
    upload(m.rowptr, m.rowptr_h);
    upload(m.col, m.col_h);
    upload(m.diag, m.diag_h);
    // ELL view (column-major), padded with self-references of slot -1
    int W = 0;
    for (int64_t i = 0; i < m.n; ++i) W = std::max(W, m.rowptr_h[i + 1] - m.rowptr_h[i]);
    m.ell_W = W;
    std::vector<int32_t> ec((size_t)W * m.n), es((size_t)W * m.n);
    for (int64_t i = 0; i < m.n; ++i)
        for (int w = 0; w < W; ++w) {
            int32_t sl = m.rowptr_h[i] + w;
            bool real = sl < m.rowptr_h[i + 1];
            ec[(size_t)w * m.n + i] = real ? m.col_h[sl] : (int32_t)i;
            es[(size_t)w * m.n + i] = real ? sl : -1;
            m.ell_bw = std::max(m.ell_bw, (int)std::abs(ec[(size_t)w * m.n + i] - (int32_t)i));
        }
    upload(m.ell_col, ec);
    upload(m.ell_slot, es);
}

// One refinement step fine -> coarse as P with <= 2 entries per fine dof, and P^T.
static void build_parent_transfer(mg_ctx* c, int fine, int coarse, const std::vector<int32_t>& parent) {
    MeshLevel& mf = c->meshes[fine];
    const MeshLevel& mc = c->meshes[coarse];
    std::vector<int32_t> par(2 * mf.n, -1);
    std::vector<float> pw(2 * mf.n, 0.0f);
    std::vector<std::vector<std::pair<int32_t, float>>> rows(mc.n);
    for (int64_t i = 0; i < mf.n; ++i) {
        int32_t v = mf.dof2node[i];
        int32_t a = parent[2 * v], b = parent[2 * v + 1];
        if (a == b) {
            par[i] = mc.node2dof[a];
            pw[i] = 1.0f;
        } else {
            par[i] = mc.node2dof[a];
            par[mf.n + i] = mc.node2dof[b];
            pw[i] = 0.5f;
            pw[mf.n + i] = 0.5f;
        }
        for (int q = 0; q < 2; ++q) {
            int32_t cd = par[q * mf.n + i];
            if (cd >= 0) rows[cd].push_back({(int32_t)i, pw[q * mf.n + i]});
            else pw[q * mf.n + i] = 0.0f;
        }
    }
    // P^T in ELL form over the coarse dofs (column-major, padded with weight 0)
    int RW = 1;
    for (auto& r : rows) RW = std::max(RW, (int)r.size());
    std::vector<int32_t> rc((size_t)RW * mc.n, 0);
    std::vector<float> rw((size_t)RW * mc.n, 0.0f);
    for (int64_t cd = 0; cd < mc.n; ++cd)
        for (size_t q = 0; q < rows[cd].size(); ++q) {
            rc[q * mc.n + cd] = rows[cd][q].first;
            rw[q * mc.n + cd] = rows[cd][q].second;
        }
    upload(mf.par, par);
    upload(mf.pw, pw);
    upload(mf.rt_col, rc);
    upload(mf.rt_w, rw);
    mf.rt_W = RW;
    mf.parent_mesh = coarse;
}

static void assemble_mesh(mg_ctx* c, MeshLevel& m) {
    build_pattern(m);
    const int64_t nt = m.n_tri;
    std::vector<double> sig(nt), nu(nt), kk(3 * nt);
    std::vector<int32_t> law(nt), esrc(nt);
    m.n_nl = 0;
    for (int64_t e = 0; e < nt; ++e) {
        int r = m.region[e];
        const Material& mt = c->mats[r];
        if (!mt.set) mg_fail(MG_ESTATE, "no material set for region " + std::to_string(r));
        sig[e] = mt.sigma;
        nu[e] = mt.nu;
        law[e] = mt.law;
        kk[3 * e] = mt.k1;
        kk[3 * e + 1] = mt.k2;
        kk[3 * e + 2] = mt.k3;
        if (mt.law == 1) m.n_nl++;
        const Source& s = c->srcs[r];
        esrc[e] = s.phase < 0 ? -1 : 2 * s.phase + (s.sign < 0 ? 1 : 0);
    }
    upload(m.elem_sigma, sig);
    upload(m.elem_nu, nu);
    upload(m.elem_law, law);
    upload(m.elem_k, kk);
    upload(m.elem_phase, esrc);
    upload(m.tri_d, m.tri);
    upload(m.xy_d, m.xy);
    m.area.ensure(nt * sizeof(double));
    m.grad.ensure(6 * nt * sizeof(double));
    m.elemK.ensure(9 * nt * sizeof(double));
    m.elemM.ensure(9 * nt * sizeof(double));
    m.K.ensure(m.nnz * sizeof(double));
    m.M.ensure(m.nnz * sizeof(double));
    m.F.ensure(3 * m.n * sizeof(double));
    clear_flag(c);
    cudaStream_t s = c->stream;
    k_elem_geometry<<<nblk(nt), 256, 0, s>>>(nt, m.tri_d.as<int32_t>(), m.xy_d.as<double>(), m.area.as<double>(),
                                            m.grad.as<double>(), c->flag.as<int>());
    k_elem_linear<<<nblk(nt), 256, 0, s>>>(nt, m.area.as<double>(), m.grad.as<double>(), m.elem_sigma.as<double>(),
                                          m.elem_nu.as<double>(), m.elemK.as<double>(), m.elemM.as<double>());
    k_gather_slots<<<nblk(m.nnz), 256, 0, s>>>(m.nnz, m.slot_ptr.as<int32_t>(), m.slot_src.as<int32_t>(),
                                              m.elemK.as<double>(), m.K.as<double>());
    k_gather_slots<<<nblk(m.nnz), 256, 0, s>>>(m.nnz, m.slot_ptr.as<int32_t>(), m.slot_src.as<int32_t>(),
                                              m.elemM.as<double>(), m.M.as<double>());
    k_phase_loads<<<nblk(m.n), 256, 0, s>>>(m.n, m.load_ptr.as<int32_t>(), m.load_src.as<int32_t>(),
                                           m.elem_phase.as<int32_t>(), m.area.as<double>(), m.F.as<double>());
    MG_CUDA(cudaGetLastError());
    if (read_flag(c)) mg_fail(MG_EINVAL, "mesh has a clockwise or degenerate triangle");
    m.assembled = true;
}

void ctx_finalize(mg_ctx* c) {
    if (c->finalized) return;
    if (c->meshes.empty()) mg_fail(MG_ESTATE, "no mesh added");
    for (auto& m : c->meshes)
        if (!m.assembled) assemble_mesh(c, m);
    for (auto& r : c->refinements)
        if (c->meshes[r.first.first].parent_mesh != r.first.second)
            build_parent_transfer(c, r.first.first, r.first.second, r.second);
    c->finalized = true;
}

static MgDepth* build_depth(mg_ctx* c, int mesh, double dt) {
    MeshLevel& m = c->meshes[mesh];
    auto* d = new MgDepth();
    d->mesh = mesh;
    d->n = m.n;
    d->W = m.ell_W;
    const int64_t nW = (int64_t)m.ell_W * m.n;
    d->L64.ensure(nW * sizeof(double));
    d->M64.ensure(nW * sizeof(double));
    d->L32.ensure(nW * sizeof(float));
    d->Llo32.ensure(nW * sizeof(float));
    d->M32.ensure(nW * sizeof(float));
    d->Mlo32.ensure(nW * sizeof(float));
    d->LD32.ensure(nW * sizeof(float));
    d->dinv64.ensure(m.n * sizeof(double));
    d->dinv32.ensure(m.n * sizeof(float));
    cudaStream_t s = c->stream;
    k_ell_values<<<nblk(nW), 256, 0, s>>>(nW, m.ell_slot.as<int32_t>(), m.K.as<double>(), m.M.as<double>(), 1.0 / dt,
                                         d->L64.as<double>(), d->M64.as<double>(), d->L32.as<float>(),
                                         d->Llo32.as<float>(), d->M32.as<float>(), d->Mlo32.as<float>());
    k_ell_diag<<<nblk(m.n), 256, 0, s>>>(m.n, m.ell_W, m.ell_col.as<int32_t>(), d->L64.as<double>(),
                                        d->dinv64.as<double>(), d->dinv32.as<float>(), c->flag.as<int>());
    k_ell_scaled<<<nblk(nW), 256, 0, s>>>(nW, m.n, m.ell_col.as<int32_t>(), d->L64.as<double>(),
                                         d->dinv64.as<double>(), d->LD32.as<float>());
    DBuf bound;
    bound.ensure(sizeof(unsigned));
    MG_CUDA(cudaMemsetAsync(bound.p, 0, sizeof(unsigned), s));
    k_ell_gershgorin<<<nblk(m.n), 256, 0, s>>>(m.n, m.ell_W, d->L64.as<double>(), d->dinv64.as<double>(),
                                               bound.as<unsigned>());
    MG_CUDA(cudaGetLastError());
    unsigned bits = 0;
    MG_CUDA(cudaMemcpyAsync(&bits, bound.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    std::memcpy(&d->lam, &bits, sizeof(float));
    return d;
}

void smoother_weights(double lam, const mg_solver_opts& so, int nu, float* w) {
    const double omega = so.omega > 0.0 ? so.omega : 0.7;
    const bool cheb = so.smoother == MG_SMOOTH_CHEBYSHEV && lam > 0.0;
    const double b = lam, a = b / (so.cheb_ratio > 0.0 ? so.cheb_ratio : 30.0);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < nu; ++k) {
        // k-th root of the first-kind Chebyshev polynomial of degree nu mapped to [a, b]
        const double theta = 0.5 * (b + a) + 0.5 * (b - a) * std::cos(pi * (2 * k + 1) / (2.0 * nu));
        w[k] = cheb ? (float)(1.0 / theta) : (float)omega;
    }
}

// Dense FP32 inverse of M/dt + K on a small base mesh (Gauss-Jordan on [A | I]
// in FP64; the operator is SPD, so no pivoting is needed).
static void build_base_inverse(mg_ctx* c, StepOp& o, int mesh, double dt) {
    MeshLevel& m = c->meshes[mesh];
    const int64_t n = m.n;
    DBuf aug, buf;
    aug.ensure((size_t)n * 2 * n * sizeof(double));
    buf.ensure((size_t)6 * n * sizeof(double));
    cudaStream_t s = c->stream;
    MG_CUDA(cudaMemsetAsync(aug.p, 0, (size_t)n * 2 * n * sizeof(double), s));
    k_dense_aug<<<nblk(n), 256, 0, s>>>(n, m.rowptr.as<int32_t>(), m.col.as<int32_t>(), m.K.as<double>(),
                                       m.M.as<double>(), 1.0 / dt, aug.as<double>());
    int dev = 0, nsm = 0, per_sm = 0;
    MG_CUDA(cudaGetDevice(&dev));
    MG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_sweep, 256, 0));
    if (per_sm < 1) mg_fail(MG_ECUDA, "Gauss-Jordan sweep cannot be resident");
    unsigned grid = (unsigned)std::min<int64_t>((int64_t)nsm * per_sm, n);
    double* aug_p = aug.as<double>();
    double* col_p = buf.as<double>();
    double* row_p = col_p + 2 * n;
    int* flag_p = c->flag.as<int>();
    int64_t n_arg = n;
    void* args[] = {&n_arg, &aug_p, &col_p, &row_p, &flag_p};
    MG_CUDA(cudaLaunchCooperativeKernel((const void*)k_gj_sweep, dim3(grid), dim3(256), args, 0, s));
    o.base_inv.ensure((size_t)n * n * sizeof(float));
    k_gj_extract<<<nblk(n * n), 256, 0, s>>>(n, aug.as<double>(), o.base_inv.as<float>());
    MG_CUDA(cudaGetLastError());
    MG_CUDA(cudaStreamSynchronize(s));
}

StepOp& ctx_step_op(mg_ctx* c, int mesh, double dt) {
    ctx_finalize(c);
    for (auto* o : c->ops)
        if (o->mesh == mesh && o->dt == dt) return *o;
    auto* o = new StepOp();
    c->ops.push_back(o);
    o->mesh = mesh;
    o->dt = dt;
    clear_flag(c);
    int cur = mesh;
    while (true) {
        o->mg.push_back(build_depth(c, cur, dt));
        int par = c->meshes[cur].parent_mesh;
        if (par < 0 || (int)o->mg.size() == MG_MAX_DEPTH) break;
        cur = par;
    }
    if (c->meshes[cur].n <= MG_MAX_DENSE) build_base_inverse(c, *o, cur, dt);
    if (read_flag(c)) {
        c->ops.pop_back();
        delete o;
        mg_fail(MG_ENOTSPD, "M/dt + K is not SPD (non-positive diagonal or pivot)");
    }
    return *o;
}

const StepOp* ctx_find_step_op(const mg_ctx* c, int mesh, double dt) {
    if (!c->finalized) return nullptr;
    for (auto* o : c->ops)
        if (o->mesh == mesh && o->dt == dt) return o;
    return nullptr;
}

const int8_t* ctx_find_pwm_table(const mg_ctx* c, int64_t N, double T) {
    return (c->pwm_N == N && c->pwm_T == T) ? c->pwm_table.as<int8_t>() : nullptr;
}

const int8_t* ctx_pwm_table(mg_ctx* c, int64_t N, double T) {
    if (!c->pwm.set) mg_fail(MG_ESTATE, "mg_set_pwm was not called");
    if (c->pwm_N == N && c->pwm_T == T) return c->pwm_table.as<int8_t>();
    c->pwm_table.ensure(3 * (N + 1));
    const PwmSpec& p = c->pwm;
    double q = p.f_carrier * T;
    int64_t q_int = -1;
    if (std::fabs(q - std::round(q)) <= 1e-9 * std::max(1.0, std::fabs(q))) q_int = (int64_t)std::llround(q);
    if (q_int >= 0 && (double)q_int * (double)N > 9.0e18) q_int = -1;  // keep q * i inside int64
    const double w = 2.0 * M_PI * p.f_ref;
    const double phi1 = -2.0 * M_PI / 3.0, phi2 = -4.0 * M_PI / 3.0;
    k_pwm_table<<<nblk(N + 1), 256, 0, c->stream>>>(N, T / (double)N, w, p.mod_index, p.carrier, q_int, p.f_carrier,
                                                   phi1, phi2, c->pwm_table.as<int8_t>());
    MG_CUDA(cudaGetLastError());
    c->pwm_N = N;
    c->pwm_T = T;
    return c->pwm_table.as<int8_t>();
}

const double* ctx_find_wave_table(const mg_ctx* c, int64_t N, double T, int kind) {
    auto it = c->waves.find({{N, T}, kind});
    return it == c->waves.end() ? nullptr : it->second.as<double>();
}

const double* ctx_wave_table(mg_ctx* c, int64_t N, double T, int kind) {
    if (const double* w = ctx_find_wave_table(c, N, T, kind)) return w;
    if (!c->pwm.set) mg_fail(MG_ESTATE, "mg_set_pwm was not called");
    DBuf& b = c->waves[{{N, T}, kind}];
    b.ensure((size_t)3 * (N + 1) * sizeof(double));
    if (kind == 0) {
        const int8_t* sg = ctx_pwm_table(c, N, T);
        k_wave_pwm<<<nblk(N + 1), 256, 0, c->stream>>>(N, T / (double)N, c->t_ramp, sg, b.as<double>());
    } else {
        const PwmSpec& p = c->pwm;
        k_wave_reference<<<nblk(N + 1), 256, 0, c->stream>>>(N, T / (double)N, 2.0 * M_PI * p.f_ref, p.mod_index,
                                                            -2.0 * M_PI / 3.0, -4.0 * M_PI / 3.0, c->t_ramp,
                                                            b.as<double>());
    }
    MG_CUDA(cudaGetLastError());
    return b.as<double>();
}

// ------------------------------------------------------------------ transfers

// Node-space prolongation rows: fine node -> list of (coarse node, weight).
using Row = std::vector<std::pair<int32_t, double>>;

static std::vector<Row> one_refinement(const std::vector<int32_t>& parent, int64_t nf) {
    std::vector<Row> P(nf);
    for (int64_t i = 0; i < nf; ++i) {
        int32_t a = parent[2 * i], b = parent[2 * i + 1];
        if (a == b) P[i] = {{a, 1.0}};
        else P[i] = {{std::min(a, b), 0.5}, {std::max(a, b), 0.5}};
    }
    return P;
}

Transfer& ctx_transfer(mg_ctx* c, int fine, int coarse) {
    ctx_finalize(c);
    auto key = std::make_pair(fine, coarse);
    auto it = c->transfers.find(key);
    if (it != c->transfers.end()) return *it->second;
    // a transfer given by the caller, or the chain of refinements fine -> ... -> coarse
    auto given = c->given_P.find(key);
    std::vector<const std::vector<int32_t>*> chain;
    std::vector<int> path{fine};
    int cur = fine;
    while (given == c->given_P.end() && cur != coarse) {
        const std::vector<int32_t>* par = nullptr;
        int nxt = -1;
        for (auto& r : c->refinements)
            if (r.first.first == cur) { par = &r.second; nxt = r.first.second; break; }
        if (!par) mg_fail(MG_EINVAL, "no refinement chain from mesh " + std::to_string(fine) + " to " +
                                         std::to_string(coarse));
        chain.push_back(par);
        cur = nxt;
        path.push_back(cur);
        if (path.size() > 16) mg_fail(MG_EINVAL, "refinement chain too long or cyclic");
    }
    const MeshLevel& mf = c->meshes[fine];
    const MeshLevel& mc = c->meshes[coarse];
    // compose node-space rows: P = P_1 P_2 ... (fine first)
    std::vector<Row> P = given != c->given_P.end() ? given->second
                                                    : one_refinement(*chain[0], c->meshes[path[0]].n_nodes);
    for (size_t k = 1; k < chain.size(); ++k) {
        std::vector<Row> Pk = one_refinement(*chain[k], c->meshes[path[k]].n_nodes);
        for (auto& row : P) {
            std::map<int32_t, double> acc;
            for (auto& [j, w] : row)
                for (auto& [jj, ww] : Pk[j]) acc[jj] += w * ww;
            row.assign(acc.begin(), acc.end());
        }
    }
    auto* t = new Transfer();
    c->transfers[key] = t;
    t->fine = fine;
    t->coarse = coarse;
    t->nf = mf.n;
    t->nc = mc.n;
    std::vector<int32_t> pp(mf.n + 1, 0), pc;
    std::vector<double> pv;
    for (int64_t d = 0; d < mf.n; ++d) {
        for (auto& [cn, w] : P[mf.dof2node[d]]) {
            int32_t cd = mc.node2dof[cn];
            if (cd < 0) continue;  // Dirichlet value is zero
            pc.push_back(cd);
            pv.push_back(w);
        }
        pp[d + 1] = (int32_t)pc.size();
    }
    // transpose
    std::vector<int32_t> tp(mc.n + 1, 0), tc(pc.size());
    std::vector<double> tv(pc.size()), rowsum(mc.n, 0.0);
    for (auto cd : pc) tp[cd + 1]++;
    std::partial_sum(tp.begin(), tp.end(), tp.begin());
    std::vector<int32_t> fillp(tp.begin(), tp.end() - 1);
    for (int64_t d = 0; d < mf.n; ++d)
        for (int32_t q = pp[d]; q < pp[d + 1]; ++q) {
            int32_t cd = pc[q];
            tc[fillp[cd]] = (int32_t)d;
            tv[fillp[cd]++] = pv[q];
        }
    for (int64_t cd = 0; cd < mc.n; ++cd)
        for (int32_t q = tp[cd]; q < tp[cd + 1]; ++q) rowsum[cd] += tv[q];
    std::vector<double> rinv(mc.n);
    for (int64_t cd = 0; cd < mc.n; ++cd) rinv[cd] = 1.0 / rowsum[cd];
    // injection: fine node coinciding with each coarse node (a given transfer: the
    // fine node whose row of P is the coarse node's unit vector)
    std::vector<int32_t> inj(mc.n, -1);
    if (given != c->given_P.end()) {
        std::vector<int32_t> at(mc.n_nodes, -1);
        for (int64_t i = 0; i < mf.n_nodes; ++i)
            if (P[i].size() == 1 && P[i][0].second == 1.0) at[P[i][0].first] = (int32_t)i;
        for (int64_t cd = 0; cd < mc.n; ++cd) {
            const int32_t fnode = at[mc.dof2node[cd]];
            if (fnode < 0 || mf.node2dof[fnode] < 0) mg_fail(MG_EINVAL, "coarse node without a fine interior node");
            inj[cd] = mf.node2dof[fnode];
        }
    } else {
        std::vector<int32_t> node(mc.n_nodes);
        std::iota(node.begin(), node.end(), 0);
        for (int k = (int)chain.size() - 1; k >= 0; --k) {
            const auto& par = *chain[k];
            int64_t nfk = c->meshes[path[k]].n_nodes;
            std::vector<int32_t> inv(c->meshes[path[k + 1]].n_nodes, -1);
            for (int64_t i = 0; i < nfk; ++i)
                if (par[2 * i] == par[2 * i + 1]) inv[par[2 * i]] = (int32_t)i;
            for (auto& v : node) v = inv[v];
        }
        for (int64_t cd = 0; cd < mc.n; ++cd) {
            int32_t fnode = node[mc.dof2node[cd]];
            if (fnode < 0 || mf.node2dof[fnode] < 0) mg_fail(MG_EINVAL, "coarse node without a fine interior node");
            inj[cd] = mf.node2dof[fnode];
        }
    }
    upload(t->P_ptr, pp);
    upload(t->P_col, pc);
    upload(t->P_val, pv);
    upload(t->PT_ptr, tp);
    upload(t->PT_col, tc);
    upload(t->PT_val, tv);
    upload(t->inj, inj);
    upload(t->PT_rowsum_inv, rinv);
    return *t;
}

// ------------------------------------------------------------------ ABI

extern "C" {

mg_status mg_create(mg_ctx** out, int device, void* cuda_stream) {
    if (!out) return MG_EINVAL;
    *out = nullptr;
    mg_ctx* c = nullptr;
    try {
        c = new mg_ctx();
    } catch (...) {
        return MG_ENOMEM;
    }
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    mg_status st = guarded(c, [&] {
        int ndev = 0;
        MG_CUDA(cudaGetDeviceCount(&ndev));
        if (device < 0 || device >= ndev) mg_fail(MG_EINVAL, "no such CUDA device");
        MG_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
        c->flag.ensure(4 * sizeof(int));
    });
    if (st != MG_OK) {
        delete c;
        return st;
    }
    *out = c;
    return MG_OK;
}

void mg_destroy(mg_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    delete c;
}

const char* mg_last_error(const mg_ctx* c) { return c ? c->err.c_str() : "null context"; }

mg_status mg_set_stream(mg_ctx* c, void* s) {
    return guarded(c, [&] { c->stream = (cudaStream_t)s; });
}

mg_status mg_add_mesh(mg_ctx* c, int* level_out, int64_t n_nodes, const double* xy, int64_t n_tri,
                      const int32_t* tri, const int32_t* region, int64_t n_dir, const int32_t* dir_nodes) {
    return guarded(c, [&] {
        if (!level_out || n_nodes <= 0 || n_tri <= 0 || !xy || !tri || !region || n_dir < 0 ||
            (n_dir > 0 && !dir_nodes))
            mg_fail(MG_EINVAL, "mg_add_mesh: bad arguments");
        if (n_nodes >= INT32_MAX || 9 * n_tri >= INT32_MAX) mg_fail(MG_EINVAL, "mesh too large");
        MeshLevel m;
        m.n_nodes = n_nodes;
        m.n_tri = n_tri;
        m.xy.assign(xy, xy + 2 * n_nodes);
        m.tri.assign(tri, tri + 3 * n_tri);
        m.region.assign(region, region + n_tri);
        for (int64_t q = 0; q < 3 * n_tri; ++q)
            if (m.tri[q] < 0 || m.tri[q] >= n_nodes) mg_fail(MG_EINVAL, "triangle node index out of range");
        for (int64_t e = 0; e < n_tri; ++e)
            if (m.region[e] < 0 || m.region[e] >= MG_MAX_REGIONS) mg_fail(MG_EINVAL, "region tag out of range");
        for (int64_t q = 0; q < 2 * n_nodes; ++q)
            if (!std::isfinite(m.xy[q])) mg_fail(MG_EINVAL, "non-finite coordinate");
        std::vector<char> isdir(n_nodes, 0);
        for (int64_t q = 0; q < n_dir; ++q) {
            if (dir_nodes[q] < 0 || dir_nodes[q] >= n_nodes) mg_fail(MG_EINVAL, "Dirichlet node out of range");
            isdir[dir_nodes[q]] = 1;
        }
        m.node2dof.assign(n_nodes, -1);
        for (int64_t i = 0; i < n_nodes; ++i)
            if (!isdir[i]) {
                m.node2dof[i] = (int32_t)m.dof2node.size();
                m.dof2node.push_back((int32_t)i);
            }
        m.n = (int64_t)m.dof2node.size();
        if (m.n == 0) mg_fail(MG_EINVAL, "mesh has no unknowns");
        c->meshes.push_back(std::move(m));
        c->finalized = false;
        *level_out = (int)c->meshes.size() - 1;
    });
}

mg_status mg_add_refinement(mg_ctx* c, int fine, int coarse, const int32_t* parent) {
    return guarded(c, [&] {
        if (fine < 0 || coarse < 0 || fine >= (int)c->meshes.size() || coarse >= (int)c->meshes.size() ||
            fine == coarse || !parent)
            mg_fail(MG_EINVAL, "mg_add_refinement: bad levels");
        int64_t nf = c->meshes[fine].n_nodes, nc = c->meshes[coarse].n_nodes;
        std::vector<int32_t> par(parent, parent + 2 * nf);
        for (auto v : par)
            if (v < 0 || v >= nc) mg_fail(MG_EINVAL, "parent node out of range");
        for (auto& r : c->refinements)
            if (r.first.first == fine) mg_fail(MG_EINVAL, "mesh already has a coarse parent");
        c->refinements.push_back({{fine, coarse}, std::move(par)});
    });
}

mg_status mg_add_transfer(mg_ctx* c, int fine, int coarse, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                          const double* val) {
    return guarded(c, [&] {
        if (fine < 0 || coarse < 0 || fine >= (int)c->meshes.size() || coarse >= (int)c->meshes.size() ||
            fine == coarse || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val)))
            mg_fail(MG_EINVAL, "mg_add_transfer: bad arguments");
        const int64_t nf = c->meshes[fine].n_nodes, nc = c->meshes[coarse].n_nodes;
        if (rowptr[0] != 0 || rowptr[nf] != nnz) mg_fail(MG_EINVAL, "mg_add_transfer: rowptr must run from 0 to nnz");
        std::vector<Row> P(nf);
        std::vector<int32_t> unit_at(nc, -1);
        for (int64_t i = 0; i < nf; ++i) {
            if (rowptr[i + 1] < rowptr[i]) mg_fail(MG_EINVAL, "mg_add_transfer: rowptr must not decrease");
            for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                if (col[q] < 0 || col[q] >= nc) mg_fail(MG_EINVAL, "mg_add_transfer: column out of range");
                if (!std::isfinite(val[q])) mg_fail(MG_EINVAL, "mg_add_transfer: value not finite");
                P[i].push_back({col[q], val[q]});
            }
            if (P[i].size() == 1 && P[i][0].second == 1.0) unit_at[P[i][0].first] = (int32_t)i;
        }
        // nodal interpolation between nested node sets: every coarse node is a fine node
        for (int64_t j = 0; j < nc; ++j)
            if (unit_at[j] < 0)
                mg_fail(MG_EINVAL, "mg_add_transfer: coarse node " + std::to_string(j) +
                                       " has no fine node whose row of P is its unit vector");
        c->given_P[{fine, coarse}] = std::move(P);
        auto it = c->transfers.find({fine, coarse});  // a transfer built before is rebuilt from this one
        if (it != c->transfers.end()) {
            delete it->second;
            c->transfers.erase(it);
        }
    });
}

mg_status mg_set_material(mg_ctx* c, int32_t region, double sigma, double nu, int law, double k1, double k2,
                          double k3) {
    return guarded(c, [&] {
        if (region < 0 || region >= MG_MAX_REGIONS || !(sigma >= 0.0) || (law != 0 && law != 1))
            mg_fail(MG_EINVAL, "mg_set_material: bad arguments");
        if (law == 0 && !(nu > 0.0)) mg_fail(MG_EINVAL, "reluctivity must be positive");
        if (law == 1 && !(k1 >= 0.0 && k2 >= 0.0 && k3 > 0.0)) mg_fail(MG_EINVAL, "Brauer law needs k1,k2 >= 0, k3 > 0");
        Material& m = c->mats[region];
        m.sigma = sigma;
        m.nu = law == 0 ? nu : k1 + k3;  // linearised value at |B| = 0 for the Brauer law
        m.law = law;
        m.k1 = k1;
        m.k2 = k2;
        m.k3 = k3;
        m.set = true;
        c->finalized = false;
        for (auto& mm : c->meshes) mm.assembled = false;
        ctx_drop_plans(c);
        for (auto* o : c->ops) delete o;
        c->ops.clear();
    });
}

mg_status mg_set_source(mg_ctx* c, int32_t region, int phase, int sign) {
    return guarded(c, [&] {
        if (region < 0 || region >= MG_MAX_REGIONS || phase < 0 || phase > 2 || (sign != 1 && sign != -1))
            mg_fail(MG_EINVAL, "mg_set_source: bad arguments");
        c->srcs[region].phase = phase;
        c->srcs[region].sign = sign;
        c->finalized = false;
        for (auto& mm : c->meshes) mm.assembled = false;
    });
}

mg_status mg_set_pwm(mg_ctx* c, double J0, double f_ref, double f_carrier, int carrier, double mod_index) {
    return guarded(c, [&] {
        if (!std::isfinite(J0) || !(f_ref >= 0.0) || !(f_carrier > 0.0) || (carrier != 0 && carrier != 1) ||
            !std::isfinite(mod_index))
            mg_fail(MG_EINVAL, "mg_set_pwm: bad arguments");
        c->pwm = PwmSpec{J0, f_ref, f_carrier, mod_index, carrier, true};
        c->pwm_N = -1;
        c->waves.clear();
    });
}

mg_status mg_set_ramp(mg_ctx* c, double t_ramp) {
    return guarded(c, [&] {
        if (!(t_ramp >= 0.0) || !std::isfinite(t_ramp)) mg_fail(MG_EINVAL, "mg_set_ramp: bad arguments");
        c->t_ramp = t_ramp;
        c->waves.clear();
    });
}

mg_status mg_finalize(mg_ctx* c) {
    return guarded(c, [&] { ctx_finalize(c); });
}

int64_t mg_num_dofs(const mg_ctx* c, int level) {
    if (!c || level < 0 || level >= (int)c->meshes.size()) return -1;
    return c->meshes[level].n;
}

mg_status mg_get_operators(mg_ctx* c, int level, int64_t* nnz_out, int64_t* rowptr, int32_t* col, double* K,
                           double* M, double* F) {
    return guarded(c, [&] {
        if (level < 0 || level >= (int)c->meshes.size()) mg_fail(MG_EINVAL, "no such mesh level");
        ctx_finalize(c);
        MeshLevel& m = c->meshes[level];
        if (nnz_out) *nnz_out = m.nnz;
        if (rowptr)
            for (int64_t i = 0; i <= m.n; ++i) rowptr[i] = m.rowptr_h[i];
        if (col) std::memcpy(col, m.col_h.data(), m.nnz * sizeof(int32_t));
        if (K) MG_CUDA(cudaMemcpyAsync(K, m.K.p, m.nnz * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (M) MG_CUDA(cudaMemcpyAsync(M, m.M.p, m.nnz * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (F) MG_CUDA(cudaMemcpyAsync(F, m.F.p, 3 * m.n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        MG_CUDA(cudaStreamSynchronize(c->stream));
    });
}

mg_status mg_pwm_table(mg_ctx* c, int64_t N, double T, int8_t* out) {
    return guarded(c, [&] {
        if (N <= 0 || !(T > 0.0) || !out) mg_fail(MG_EINVAL, "mg_pwm_table: bad arguments");
        const int8_t* d = ctx_pwm_table(c, N, T);
        MG_CUDA(cudaMemcpyAsync(out, d, 3 * (N + 1), cudaMemcpyDeviceToHost, c->stream));
        MG_CUDA(cudaStreamSynchronize(c->stream));
    });
}

}  // extern "C"

// used by the solver translation units
mg_status mg_guarded_call(mg_ctx* c, void (*fn)(void*), void* arg) {
    return guarded(c, [&] { fn(arg); });
}
