// Internal state of libmgrit_em.so (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "mgrit_em.h"

#define MG_MAX_REGIONS 64
#define MG_MAX_DEPTH 6
#define MG_MAX_DENSE 4096   // largest base mesh inverted densely
#define MG_MAX_NU 8         // smoothing sweeps per side of the V-cycle

struct MgError {
    mg_status st;
    std::string msg;
};

// Throw from host code inside the library; every ABI entry point catches.
[[noreturn]] void mg_fail(mg_status st, const std::string& msg);
void mg_check_cuda(cudaError_t e, const char* what);
#define MG_CUDA(call) mg_check_cuda((call), #call)

// Device buffer owned by the context.
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void release();
    void ensure(size_t nbytes);  // grow (contents not kept)
    template <class T> T* as() const { return static_cast<T*>(p); }
};

template <class T>
void upload(DBuf& b, const std::vector<T>& v) {
    b.ensure(v.size() * sizeof(T));
    if (!v.empty()) MG_CUDA(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

struct Material {
    double sigma = 0.0, nu = 0.0;
    int law = 0;
    double k1 = 0.0, k2 = 0.0, k3 = 0.0;
    bool set = false;
};

struct Source {
    int phase = -1, sign = 0;
};

struct PwmSpec {
    double J0 = 0.0, f_ref = 50.0, f_carrier = 5e3, mod_index = 1.0;
    int carrier = 1;
    bool set = false;
};

// One P1 mesh and its assembled linear operators (interior unknowns only).
struct MeshLevel {
    int64_t n_nodes = 0, n_tri = 0, n = 0, nnz = 0;
    int64_t n_nl = 0;           // elements with a nonlinear material law
    std::vector<double> xy;
    std::vector<int32_t> tri, region;
    std::vector<int32_t> node2dof;  // -1 on Dirichlet nodes
    std::vector<int32_t> dof2node;
    // CSR pattern of the interior block (host copies)
    std::vector<int32_t> rowptr_h, col_h, diag_h;
    // device data
    DBuf rowptr, col, diag;     // int32
    DBuf tri_d, xy_d;           // int32 / double
    DBuf slot_ptr, slot_src;    // slot -> element-local contributions (elem * 9 + a * 3 + b)
    DBuf load_ptr, load_src;    // dof -> element-local vertex contributions (elem * 3 + a)
    DBuf elem_sigma, elem_nu, elem_law, elem_k, elem_phase;  // per-element material data
    DBuf area, grad;            // |T| and barycentric gradients (6 per element)
    DBuf elemK, elemM;          // 9 values per element
    DBuf K, M, F;               // nnz, nnz, 3 * n (double)
    // ELL view of the CSR pattern: width W, column-major (entry w of row i at w * n + i);
    // padding entries point at the row itself with slot -1
    int ell_W = 0;
    int ell_bw = 0;             // bandwidth max |i - j| over the pattern (padding included)
    DBuf ell_col, ell_slot;     // int32 W x n
    // one refinement step to the coarse parent mesh (if any): P with <= 2 entries per fine row
    int parent_mesh = -1;
    DBuf par, pw;               // int32 2 x n coarse dofs (-1: none), float 2 x n weights
    int rt_W = 0;
    DBuf rt_col, rt_w;          // P^T as ELL (rt_W x n_parent, column-major) over the parent's dofs
    bool assembled = false;
};

// One level of the multigrid hierarchy of a step operator (same dt on every level).
struct MgDepth {
    int mesh = 0;
    int64_t n = 0;
    int W = 0;
    DBuf L64, M64, L32, LD32, dinv64, dinv32;  // ELL values (W x n) and Jacobi data
    DBuf Llo32;  // L64 - L32 rounded to FP32: L32 + Llo32 carries L64 to about 2^-48
    DBuf M32, Mlo32;  // the same two-part FP32 form of M64
    float lam = 0.0f;  // Gershgorin bound of the spectrum of D^-1 L (rounded up)
};

// L = M / dt + K on one mesh level and its multigrid hierarchy: depth 0 is the
// level itself, depth d+1 the parent mesh of depth d, the last depth the base mesh
// (no parent), solved by the dense inverse `base_inv` (FP32, n x n row-major).
struct StepOp {
    int mesh = 0;
    double dt = 0.0;
    std::vector<MgDepth*> mg;
    DBuf base_inv;
    ~StepOp() { for (auto* d : mg) delete d; }
};

// P_s between two mesh levels (composed over refinements), interior DOFs.
struct Transfer {
    int fine = -1, coarse = -1;
    int64_t nf = 0, nc = 0;
    DBuf P_ptr, P_col, P_val;    // CSR n_f x n_c
    DBuf PT_ptr, PT_col, PT_val; // CSR n_c x n_f
    DBuf inj;                    // n_c: fine dof at each coarse dof's node
    DBuf PT_rowsum_inv;          // n_c: 1 / (P^T 1)
};

struct GraphPlan;
void graph_plan_delete(GraphPlan* p);
struct NewtonPlan;
void newton_plan_delete(NewtonPlan* p);
struct NlMesh;
void nl_mesh_delete(NlMesh* p);

struct mg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;
    std::vector<MeshLevel> meshes;
    std::vector<std::pair<std::pair<int, int>, std::vector<int32_t>>> refinements;  // (fine, coarse) -> parent
    // transfers given as node-space CSR matrices (mg_add_transfer): (fine, coarse) -> rows
    std::map<std::pair<int, int>, std::vector<std::vector<std::pair<int32_t, double>>>> given_P;
    Material mats[MG_MAX_REGIONS];
    Source srcs[MG_MAX_REGIONS];
    PwmSpec pwm;
    bool finalized = false;
    std::vector<StepOp*> ops;
    std::map<std::pair<int, int>, Transfer*> transfers;
    // PWM table cache
    DBuf pwm_table;
    int64_t pwm_N = -1;
    double pwm_T = 0.0;
    // source waveform tables per (N, T, kind): kind 0 PWM signs, 1 sine reference,
    // both times the start-up ramp over the first t_ramp seconds (0: none)
    double t_ramp = 0.0;
    std::map<std::pair<std::pair<int64_t, double>, int>, DBuf> waves;
    // reusable workspaces
    DBuf ws[32];       // step-solver work vectors
    DBuf host_in, host_out;  // staging of the *_host entry points
    DBuf counters;     // device: [u64 PCG iteration sum][i32 worst status]
    DBuf flag;         // int32 error flag
    DBuf solve_buf[16];  // MGRIT level storage
    std::vector<GraphPlan*> plans;  // graph-path step plans (buffers + instantiated graphs)
    std::vector<NewtonPlan*> nplans;  // Newton-step plans (own their per-column PCG graphs)
    std::map<int, NlMesh*> nl;       // mesh -> static data of its nonlinear elements
    struct Shape {                   // launch shape chosen by mg_autotune
        int path, tile, cluster, rbs0, rbs1, base_tiles, hf, bc;
        double ms;
    };
    std::map<std::pair<int, int>, Shape> tuned;  // (mesh, column bucket) -> shape
    ~mg_ctx();
};


// ---- set-up helpers (setup.cu)
void ctx_finalize(mg_ctx* c);
StepOp& ctx_step_op(mg_ctx* c, int mesh, double dt);
Transfer& ctx_transfer(mg_ctx* c, int fine, int coarse);
const int8_t* ctx_pwm_table(mg_ctx* c, int64_t N, double T);
const double* ctx_wave_table(mg_ctx* c, int64_t N, double T, int kind);
// Lookups that never allocate: null if the operator / PWM table was not built yet.
const StepOp* ctx_find_step_op(const mg_ctx* c, int mesh, double dt);
// Weights of the nu smoothing sweeps of one pre-smoothing (post-smoothing takes them
// in reverse order): reciprocal Chebyshev roots on [lam / ratio, lam] when the
// options ask for Chebyshev smoothing and lam > 0, else omega.
void smoother_weights(double lam, const mg_solver_opts& so, int nu, float* w);
inline int smooth_sweeps(const mg_solver_opts& so) { return so.smooth > 0 ? so.smooth : 5; }
const int8_t* ctx_find_pwm_table(const mg_ctx* c, int64_t N, double T);
const double* ctx_find_wave_table(const mg_ctx* c, int64_t N, double T, int kind);

// Rounding floor of a step's FP64 residual.  One row of r = b - L x with W stored
// entries is a sum of W + 1 products; its computed value differs from the exact one
// by at most gamma_{W+1} (|b_i| + sum_j |L_ij| |x_j|), gamma_k = k u / (1 - k u),
// u = 2^-53 (the standard bound for recursive summation of products).  A column
// whose computed ||r|| is within a small multiple of gamma_{W+1} S,
// S = || |b| + |L| |x| ||, solves its step to working precision: the PCG iteration
// stops at gamma S, and an initial guess (or a refined iterate) is accepted as it is
// up to kFloorAccept gamma S, which covers the gap between the recurrence residual
// and the true residual that a finished solve leaves.  With the guess accepted,
// re-solving a step from its own solution returns that solution bit for bit.
// S is a magnitude estimate, formed in FP32 from the FP32 operator and |x| (so
// that it costs no FP64 arithmetic); its relative error, ~1e-7, does not matter.
inline double residual_floor(int W) {
    const double u = 1.1102230246251565e-16;  // 2^-53
    const double k = (double)(W + 1);
    return k * u / (1.0 - k * u);
}
constexpr double kFloorAccept = 4.0;
// FP32+refinement: FP32 PCG iterations after which a column's FP64 residual is
// recomputed even if its FP32 residual has not fallen by inner_tol (the FP32
// recurrence of a stiff step stops tracking the true residual after 2-3 orders)
constexpr int kMaxInner = 10;

// Reject solver options outside their documented ranges (MG_EINVAL); every entry
// point that runs a step calls it before any launch (mgrit.cu).
void check_solver_opts(const mg_solver_opts& so);

// ---- batched backward-Euler step (pcg.cu)
struct PhiIO {
    int k = 0;
    const double* xprev = nullptr;
    int64_t ld_prev = 0;
    const double* g = nullptr;  // added after the solve (FAS right-hand side), may be null
    int64_t ld_g = 0;
    const double* guess = nullptr;  // initial guess of Phi(xprev) + g, may be null
    int64_t ld_guess = 0;
    double* xout = nullptr;
    int64_t ld_out = 0;
    const double* wave = nullptr;   // (N+1) x 3 source waveform of the fine grid (PWM signs x ramp, or reference)
    int64_t t0 = 0, tstride = 0;    // fine time index of column c: t0 + c * tstride
};

struct SolveCounters {
    int64_t step_solves = 0, batched_steps = 0, cg_iters = 0, launches = 0, newton_iters = 0;
    int32_t worst_status = 0;
};

// Enqueue one batched step (no synchronisation).  PCG iteration totals and the
// worst per-column status accumulate in ctx->counters on the device;
// `counters` (host, may be null) counts launches and column-steps.
void phi_batch(mg_ctx* c, const StepOp& op, const PhiIO& io, const mg_solver_opts& so,
               SolveCounters* counters);
// Graph path (batch.cu): one kernel per phase over all tiles, loop in a CUDA graph.
void phi_batch_graph(mg_ctx* c, const StepOp& op, const PhiIO& io, const mg_solver_opts& so,
                     SolveCounters* counters);
void ctx_drop_plans(mg_ctx* c);
// Diagnostics on stderr, from the environment variable MGRIT_EM_TRACE: 0 off,
// 1 one line per MGRIT iteration, 2 also one line per batched Newton step, 3 also
// one line per autotuner trial (each trial then synchronises the stream).
int mg_trace_level();
// column bucket of the autotuner's table: k itself up to 16, else whole 16-column tiles
inline int tune_bucket(int k) { return k <= 16 ? k : (k + 15) / 16 * 16; }

// ---- per-column systems: the graph path's PCG with one operator per column
// (tile-major storage, 16 columns per tile; see batch.cu)
constexpr int MG_TILE = 16;
struct PcDepth {
    double* J64 = nullptr;   // depth 0 only: FP64 operator of the PCG
    float* J32 = nullptr;    // FP32 operator of the V-cycle
    float* LD32 = nullptr;   // J32 scaled by the column's 1/diag of the neighbour row
    float* dinv32 = nullptr; // 1/diag per row and column
};
struct PcOperator {
    PcDepth d[MG_MAX_DEPTH];
    const float* band_L = nullptr;  // banded Cholesky factor of the base depth per column
    const float* band_U = nullptr;
    int band_u = 0, band_stride = 0;
    const double* R = nullptr;      // residual: the system solved is J delta = -R
    const int* state = nullptr;     // only columns with state 1 are solved
    // per depth, device: Gershgorin bound of D^-1 J over all columns (float bits),
    // refreshed with every Jacobian; the plan's Chebyshev weights are divided by it
    const unsigned* lam = nullptr;
};
GraphPlan* graph_plan_pc(mg_ctx* c, const StepOp& op, int ntile, const mg_solver_opts& so, const PcOperator& pco);
double* graph_plan_solution(GraphPlan* p);
void graph_plan_run(mg_ctx* c, GraphPlan* p, int k, const mg_solver_opts& so);

// ---- the coarsening planner's probe (mgrit.cu): `iters` MGRIT iterations from
// a0 = 0 with opts (tolerance ignored); residual history and solve seconds
void mgrit_probe(mg_ctx* c, int64_t N, double T, const mg_opts& opts, int iters, std::vector<double>& hist,
                 double& seconds);

// ---- Newton steps for meshes with nonlinear materials (newton.cu)
bool mesh_is_nonlinear(const mg_ctx* c, int mesh);
void phi_batch_newton(mg_ctx* c, const StepOp& op, const PhiIO& io, const mg_solver_opts& so,
                      SolveCounters* counters);
