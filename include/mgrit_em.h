/*
 * mgrit_em.h -- C ABI of the GB300 MGRIT eddy-current library (libmgrit_em.so).
 *
 * The library solves the semi-discrete 2D eddy-current problem
 *     M a'(t) + K(a) a = f(t),   f(t) = J0 * sum_s b_s(t) F_s          (Sec. 3.1,
 *                                                   Eq. semi_discrete_system)
 * on P1 triangle meshes, with backward Euler (Eq. discrete_system) as the
 * one-step propagator Phi (Sec. 2, Eq. mgrit_nonlinear_system), either
 * sequentially (forward block solve of the block-bidiagonal space-time system,
 * Sec. 2) or by FAS-MGRIT (Algorithm 1, Sec. 2.1) with F/FCF relaxation,
 * injection in time, ideal interpolation, and spatial coarsening between
 * nested meshes (Sec. 2.2, Sec. 3.4).  b_s(t) is the three-phase PWM switching
 * function (Sec. 3.2-3.3, Eqs. machine_pwm, machine_reference_signal,
 * machine_carrier_signal).
 *
 * Conventions
 *  - Every call returns mg_status; no C++ exception crosses the ABI.  On error
 *    mg_last_error() holds a message (valid until the next call on that context).
 *  - Set-up calls take HOST arrays and copy them; the caller keeps ownership.
 *  - Solve calls take DEVICE pointers (e.g. torch CUDA tensors) unless the
 *    function name ends in _host.  The library never frees caller memory.
 *  - Vectors of one mesh level hold its interior nodes (Dirichlet A_z = 0 nodes
 *    removed) in increasing node order.  A trajectory is time-major:
 *    out[i * n + j] = a_j(t_i), i = 0..N.  A batch of k vectors is node-major:
 *    x[j * ld + c] is node j of column c (ld >= k).
 *  - Work is enqueued on the context's stream; calls that return statistics
 *    synchronise that stream.
 *  - Invalid arguments are rejected with MG_EINVAL before any launch.
 *  - Solver failures (CG or Newton not converged, MGRIT max iterations) are
 *    reported as a status; the outputs then hold the last iterate.
 *  - Every device wait inside the library's kernels is bounded; a wait that
 *    runs out returns MG_ETIMEOUT instead of hanging.
 */
#ifndef MGRIT_EM_H
#define MGRIT_EM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx;

typedef enum {
    MG_OK = 0,
    MG_EINVAL = -1,        /* bad argument, size or index                       */
    MG_ENOMEM = -2,        /* device or host allocation failed                  */
    MG_ECUDA = -3,         /* a CUDA runtime call failed                        */
    MG_ENOTSPD = -4,       /* an assembled operator is not SPD (non-positive pivot) */
    MG_ECG_MAXIT = -5,     /* a linear solve hit its iteration limit            */
    MG_ENEWTON = -6,       /* Newton did not converge (Sec. 5: poor initial guess) */
    MG_EMGRIT_MAXIT = -7,  /* MGRIT reached max_iter before the tolerance       */
    MG_ETIMEOUT = -8,      /* a bounded device wait ran out                     */
    MG_ESTATE = -9,        /* call order violated (e.g. solve before set-up)    */
    MG_ESTALLED = -10,     /* MGRIT residual stopped decreasing above the tolerance */
    MG_ENONFINITE = -11    /* a step solve met a NaN or infinity (e.g. in an input state) */
} mg_status;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`; work goes to `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream). */
mg_status mg_create(mg_ctx** out, int device, void* cuda_stream);
void mg_destroy(mg_ctx* ctx);
const char* mg_last_error(const mg_ctx* ctx);
mg_status mg_set_stream(mg_ctx* ctx, void* cuda_stream);

/* ------------------------------------------------------------------- set-up */

/* Add a P1 triangle mesh (Sec. 3.4).  xy: 2*n_nodes doubles (x, y per node);
 * tri: 3*n_tri node ids, counter-clockwise; region: n_tri tags in [0, 64);
 * dir_nodes: the n_dir nodes with A_z = 0 (the other nodes are the unknowns).
 * *level_out receives the mesh level id (0, 1, ... in call order). */
mg_status mg_add_mesh(mg_ctx* ctx, int* level_out, int64_t n_nodes, const double* xy,
                      int64_t n_tri, const int32_t* tri, const int32_t* region,
                      int64_t n_dir, const int32_t* dir_nodes);

/* Nested refinement between two added meshes (Sec. 3.4: FE nodal interpolation
 * as grid transfer).  parent: 2 * n_nodes(fine) coarse node ids; a fine node
 * with equal parents coincides with that coarse node, otherwise it is the
 * midpoint of the coarse edge (p0, p1).  Defines P_s (fine <- coarse) between
 * the two levels; transfers across several refinements are composed. */
mg_status mg_add_refinement(mg_ctx* ctx, int fine_level, int coarse_level, const int32_t* parent);

/* Spatial transfer between two added meshes given as a matrix (Sec. 3.4: FE nodal
 * interpolation P_s from the coarse to the fine mesh, Algorithm 1's interpolation;
 * Sec. 2.2 spatial coarsening).  P is node-indexed CSR over ALL nodes (Dirichlet
 * ones included): rowptr[n_nodes(fine) + 1] (int64, rowptr[0] = 0, rowptr[end] =
 * nnz), col[nnz] coarse node ids, val[nnz] weights; host arrays, copied.  The node
 * sets must be nested: every coarse node has a fine node whose row of P is that
 * coarse node's unit vector (one entry, weight exactly 1); MGRIT restricts states by
 * injection at those nodes and residuals by P^T as restrict_mode says.  Meshes need
 * not come from red refinement (e.g. a barycentric split).  For MGRIT levels on the
 * pair (fine, coarse) this matrix replaces a transfer composed from refinements;
 * the step solver's multigrid preconditioner still uses refinements only.
 * MG_EINVAL for bad levels, indices, non-finite weights or non-nested node sets. */
mg_status mg_add_transfer(mg_ctx* ctx, int fine_level, int coarse_level, int64_t nnz, const int64_t* rowptr,
                          const int32_t* col, const double* val);

/* Material of a region tag (Sec. 3.1; Sec. 5 for the Brauer law):
 * law 0: nu constant; law 1: nu(|B|^2) = k1 exp(k2 |B|^2) + k3 (nu unused). */
mg_status mg_set_material(mg_ctx* ctx, int32_t region, double sigma, double nu, int law,
                          double k1, double k2, double k3);

/* Region `region` carries J_s = sign * J0 * b_phase(t) (phase 0..2, sign +-1). */
mg_status mg_set_source(mg_ctx* ctx, int32_t region, int phase, int sign);

/* PWM source (Sec. 3.2-3.3): b_s = sgn(r_s - c), sgn(0) = 0,
 * r_s = mod_index sin(2 pi f_ref t + phi_s), phi = (0, -2pi/3, -4pi/3);
 * carrier 0: sawtooth 2 frac(f_c t) - 1 (Eq. machine_carrier_signal);
 * carrier 1: triangle 1 - 4 |frac(f_c t) - 1/2|.  t_i = i T / N; when f_c T is
 * an integer the carrier phase is formed exactly from integers. */
mg_status mg_set_pwm(mg_ctx* ctx, double J0, double f_ref, double f_carrier, int carrier,
                     double mod_index);

/* Start-up ramp of the source (Sec. 3.3, used with the nonlinear law): the
 * source waveform is multiplied by 0.5 (1 - cos(pi t / t_ramp)) for t < t_ramp
 * (the paper's two electric periods: t_ramp = 2 / f_ref); 0 switches it off (the
 * default).  Applies to the PWM source and to the sine reference. */
mg_status mg_set_ramp(mg_ctx* ctx, double t_ramp);

/* Assemble all meshes (P1 stiffness, consistent mass, phase loads) on the device.
 * Called implicitly by the first solve; returns MG_ENOTSPD if an operator has a
 * non-positive diagonal. */
mg_status mg_finalize(mg_ctx* ctx);

/* Number of unknowns (interior nodes) of a mesh level, or -1. */
int64_t mg_num_dofs(const mg_ctx* ctx, int level);

/* Copy the assembled operators of a level to HOST buffers (for inspection):
 * rowptr[n+1] (int64), col[nnz] (int32), K[nnz], M[nnz] (double) and
 * F[3*n] (phase-major).  Pass NULL for any output to skip it; *nnz_out
 * receives the number of stored entries. */
mg_status mg_get_operators(mg_ctx* ctx, int level, int64_t* nnz_out, int64_t* rowptr,
                           int32_t* col, double* K, double* M, double* F);

/* PWM table of the fine grid t_i = i T / N, i = 0..N, into HOST out[3*(N+1)]
 * (row i holds b_1, b_2, b_3 of t_i), computed by the library's kernel. */
mg_status mg_pwm_table(mg_ctx* ctx, int64_t N, double T, int8_t* out);

/* ---------------------------------------------------------------- solving */

typedef enum { MG_FP64 = 0, MG_FP32_REFINE = 1 } mg_precision;

typedef enum { MG_PRECOND_JACOBI = 0, MG_PRECOND_MULTIGRID = 1 } mg_precond;

/* Smoother of the multigrid V-cycle.  Both are polynomial (Richardson) sweeps
 * x += w_s D^-1 (r - L x) with the Jacobi diagonal D.  MG_SMOOTH_JACOBI: every
 * sweep has the weight omega.  MG_SMOOTH_CHEBYSHEV: the nu sweeps of a pre- (and,
 * in reverse order, post-) smoothing take as weights the reciprocals of the nu
 * roots of the first-kind Chebyshev polynomial on [lam / cheb_ratio, lam], lam
 * the Gershgorin bound max_i sum_j |L_ij| / L_ii of the depth's operator, so that
 * the sweeps together damp that whole upper part of the spectrum of D^-1 L (the
 * factors commute, so the V-cycle stays symmetric).  Newton corrections of
 * nonlinear meshes take as lam the largest such bound over the Jacobians of all
 * columns, recomputed on the device with every Jacobian. */
typedef enum { MG_SMOOTH_CHEBYSHEV = 0, MG_SMOOTH_JACOBI = 1 } mg_smoother;

/* How a batched step runs: MG_PATH_CLUSTER = one persistent launch, a thread-block
 * cluster per tile of columns (lowest latency for few columns); MG_PATH_GRAPH =
 * one kernel per phase over all columns, the iteration loop inside a CUDA graph
 * (full-GPU throughput for many columns); MG_PATH_AUTO picks the graph path from
 * MG_GRAPH_MIN_COLUMNS columns on.  Both compute the same step. */
typedef enum { MG_PATH_AUTO = 0, MG_PATH_CLUSTER = 1, MG_PATH_GRAPH = 2 } mg_path;
#define MG_GRAPH_MIN_COLUMNS 16

typedef struct {
    /* linear solver of one backward-Euler step: batched PCG, preconditioned by
     * one FP32 geometric-multigrid V-cycle over the nested meshes (coarsest mesh
     * solved by a dense inverse) or by Jacobi */
    double cg_tol;      /* FP64 mode: stop at ||b - L x|| <= cg_tol ||b|| per column      */
    double refine_tol;  /* FP32+refinement: FP64 stop ||b - L x|| <= refine_tol ||b||        */
    double inner_tol;   /* FP32+refinement: the FP32 PCG runs on across FP64 residual updates
                           (reliable updates): a column's FP64 residual b - L x is recomputed
                           once its FP32 residual has fallen by inner_tol since the last one,
                           or after 10 FP32 iterations without one                         */
    int max_cg;         /* iteration limit of one PCG (FP32+refinement: of its FP32 iterations) */
    int max_refine;     /* FP32+refinement: limit of FP64 residual updates                 */
    int precision;      /* mg_precision                                                    */
    int cluster;        /* CTAs per cluster (1..16; above 8 needs non-portable clusters), 0 = library
                           choice (16 for a single column tile when the device allows it, else 8) */
    int tile;           /* columns per cluster (1, 8, 16, 32), 0 = library choice          */
    int precond;        /* mg_precond                                                      */
    int smooth;         /* smoothing sweeps before and after each coarse correction (1..8),
                           0 = library choice (5)                                          */
    double omega;       /* MG_SMOOTH_JACOBI weight                                         */
    int path;           /* mg_path                                                         */
    /* nonlinear steps (meshes with a Brauer-law material, Sec. 5): damped Newton,
     * each correction J delta = -F solved by the PCG above (FP64 form, multigrid
     * with per-column Galerkin coarse operators and a banded base solve) */
    double newton_tol;  /* stop once ||delta|| <= newton_tol ||a + delta|| (full correction taken) */
    int max_newton;     /* Newton iterations per step; more is MG_ENEWTON                   */
    int max_halvings;   /* step-length halvings per iteration while ||F|| would grow        */
    double newton_lin_tol; /* PCG stop of each correction: ||J delta + F|| <= newton_lin_tol ||F||
                              (an inexact Newton step; the last correction is below newton_tol,
                              so its relative error does not reach the result)               */
    /* launch shape of the graph path; 0 = library choice, or the shape mg_autotune
     * recorded in the context for this mesh and column count */
    int rows_per_block;        /* rows per block on the finest multigrid depth (16..4096)   */
    int coarse_rows_per_block; /* rows per block on the coarser depths (16..4096)           */
    int base_tiles;            /* 16-column tiles per block of the dense base solve (1, 2, 4) */
    int smoother;              /* mg_smoother                                               */
    double cheb_ratio;         /* MG_SMOOTH_CHEBYSHEV: lam over the lower end of the damped
                                  interval (1 < cheb_ratio <= 1e4), 0 = library choice (30) */
    int halo_fusion;           /* graph path, linear steps: 2 = kernels that keep an
                                  intermediate vector in shared memory on a halo of the
                                  operator's bandwidth (two consecutive smoothing sweeps per
                                  launch; the prolongation with the residual update), where the
                                  halo fits; 3 = as 2, and the sweeps' input vector is staged
                                  in shared memory too; 1 = one kernel per sweep and per
                                  transfer; 0 = library choice (2).  Same arithmetic in all. */
    int base_cores;            /* graph path, linear steps: the dense base solve x = A^-1 r of
                                  the V-cycle on MG_BASE_CUDA (FP32 FMA) or MG_BASE_TENSOR
                                  (3xTF32 mma.sync, FP32-level accuracy) cores, 0 = library
                                  choice (MG_BASE_CUDA) */
} mg_solver_opts;
#define MG_BASE_CUDA 1
#define MG_BASE_TENSOR 2

/* Fill opts with the library defaults (cg_tol 1e-13, refine_tol 1e-13,
 * inner_tol 3e-2, max_cg 2000, max_refine 30, FP64, multigrid with 5 Chebyshev
 * sweeps on [lam/30, lam] before and after each coarse correction (omega 0.7 for
 * MG_SMOOTH_JACOBI); newton_tol 1e-8, max_newton 100,
 * max_halvings 40, newton_lin_tol 1e-6). */
void mg_solver_defaults(mg_solver_opts* opts);

/* The smoothing weights the V-cycle uses on a depth whose Gershgorin bound of
 * D^-1 L is lam (host computation, no device work, no context): w[0 .. nu-1] of
 * one pre-smoothing, post-smoothing takes them in reverse order.  With
 * MG_SMOOTH_CHEBYSHEV and lam > 0 they are the reciprocals of the roots of the
 * first-kind Chebyshev polynomial of degree nu on [lam / cheb_ratio, lam] (cheb_ratio
 * 0: 30), so that prod_s (1 - w_s x) has the smallest maximum modulus on that
 * interval among degree-nu polynomials equal to 1 at x = 0; otherwise every weight is
 * omega (0: 0.7).  w: nu floats, caller-owned.  MG_EINVAL for bad options, nu outside
 * 1..8 or lam < 0. */
mg_status mg_smoother_weights(const mg_solver_opts* opts, double lam, int nu, float* w);

typedef struct {
    int iters;                /* MGRIT iterations (coarse-grid corrections)        */
    int n_hist;               /* entries of res_hist                               */
    double res_hist[64];      /* fine-level C-point residual norm after each relaxation */
    double t_setup, t_solve;  /* seconds (host clock around synchronised phases)   */
    int64_t step_solves;      /* column-steps solved (one Phi application each)    */
    int64_t batched_steps;    /* Phi launches (each over one batch of columns)     */
    int64_t cg_iters;         /* PCG iterations summed over columns (FP32+refinement:
                                 per column tile, the inner iterations of its slowest column) */
    int32_t worst_status;     /* worst per-column solver status seen               */
    int64_t launches;         /* CUDA kernels the call launched                    */
    int64_t newton_iters;     /* Newton iterations summed over column-steps (nonlinear meshes) */
} mg_stats;

/* One batched backward-Euler step on mesh `level` (Eq. discrete_system):
 * for each column c < k, x_out[:, c] solves
 *     (M/dt + K) x = (M/dt) x_in[:, c] + J0 sum_s b_s(t_{i_c}) F_s,
 * with dt = dt_mult * T / N and fine time index i_c = i0 + c * istride
 * (0 <= i_c <= N).  x_out also serves as the initial guess when guess != 0.
 * On a mesh with a nonlinear material (Sec. 5) K depends on x and the step is
 * (M/dt)(x - x_in[:, c]) + K(x) x = J0 sum_s b_s F_s, solved by damped Newton
 * from x_in[:, c] (or from the guess); a column whose Newton iteration fails
 * reports MG_ENEWTON and keeps its last iterate.
 * Node-major layouts with leading dimensions ld_in, ld_out >= k.
 * Each column's linear solve stops at ||b - L x|| <= cg_tol ||b|| (refine_tol for
 * FP32+refinement) or at the rounding floor of its FP64 residual, whichever is
 * larger: ||b - L x|| <= gamma_{W+1} || |b| + |L| |x| ||, gamma_k = k u / (1 - k u),
 * u = 2^-53, W the stored entries per row; an initial guess within 4 gamma_{W+1}
 * of that norm is returned unchanged, so re-solving a step from its own solution
 * gives that solution back.
 * stats may be NULL; then the call does not synchronise and per-column solver
 * failures (MG_ECG_MAXIT, MG_ENEWTON) are not reported: pass stats to get them. */
mg_status mg_step(mg_ctx* ctx, int level, int64_t N, double T, int64_t dt_mult, int k,
                  int64_t i0, int64_t istride, const double* x_in, int64_t ld_in,
                  double* x_out, int64_t ld_out, int guess, const mg_solver_opts* opts,
                  mg_stats* stats);

/* mg_step without device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory at the time of the
 * call -- code being recorded into a CUDA graph by stream capture (where
 * cudaMalloc is not allowed), callers running under an external memory manager
 * or a fixed memory budget, and real-time loops that must not block in the
 * allocator.  It computes exactly what mg_step computes (no FAS term g), but its
 * work vectors live in one fixed-size array in device memory that the library
 * declares statically: 32 MiB per device, held by every GPU that loads the
 * library until the process exits.  Steps whose work vectors do not fit (about
 * 60 bytes per unknown and column in the FP64 form, 3/4 of that with
 * FP32+refinement, plus 1/3 more for the coarser multigrid levels) are rejected
 * with MG_EINVAL and a message naming the bytes needed.
 * It also allocates no operator: the step operator for (level, dt) and the PWM
 * table for (N, T) must already exist, built by one regular mg_step call with the
 * same arguments; otherwise MG_ESTATE.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents (the kernel initialises everything it reads): calls whose kernels may
 * overlap on the GPU -- other streams, other host threads -- race and must be
 * serialised by the caller.  stats may be NULL (no synchronisation). */
mg_status mg_step_static(mg_ctx* ctx, int level, int64_t N, double T, int64_t dt_mult, int k,
                         int64_t i0, int64_t istride, const double* x_in, int64_t ld_in,
                         double* x_out, int64_t ld_out, int guess, const mg_solver_opts* opts,
                         mg_stats* stats);

/* Autotuner (the paper has no counterpart): times batched linear steps of k
 * columns on mesh `level` (dt = T/N; start states are a fixed pseudo-random
 * pattern generated on the device) for a set of launch shapes -- cluster path
 * with tile width 1/8/16 and 8 or 16 CTAs per cluster, or graph path with rows
 * per block on the finest and coarser depths, halo-fused multigrid kernels or
 * not, the cores of the dense base solve and its tiles per block -- by
 * coordinate descent from the library's choice, 3 timed steps per shape.  The
 * fastest shape is written into *opts (path, tile, cluster, rows_per_block,
 * coarse_rows_per_block, halo_fusion, base_cores, base_tiles; other fields
 * kept) and recorded in the
 * context for (level, k) -- k rounded up to whole 16-column tiles above 16 --,
 * where steps with path MG_PATH_AUTO and a zero shape pick it up (MGRIT
 * relaxation batches included).  best_ms (may
 * be NULL) receives the time per step of the chosen shape.  Allocates device
 * memory for the trial vectors; synchronises.  Nonlinear meshes: MG_EINVAL. */
mg_status mg_autotune(mg_ctx* ctx, int level, int64_t N, double T, int k, mg_solver_opts* opts,
                      double* best_ms);

/* Sequential time stepping (forward block solve, Sec. 2): out[0] = a0,
 * out[i] = Phi_i(out[i-1]), i = 1..N, on mesh `level` with dt = T/N.
 * a0: n doubles; out: (N+1)*n doubles, time-major (device pointers). */
mg_status mg_sequential(mg_ctx* ctx, int level, int64_t N, double T, const double* a0,
                        double* out, const mg_solver_opts* opts, mg_stats* stats);

typedef struct {
    int levels;            /* time levels L >= 1 (1 = sequential solve)                  */
    int m[8];              /* coarsening factor from level l to l+1, l < L-1             */
    int space_level[8];    /* mesh level used on each time level (spatial coarsening)   */
    int relax;             /* 0: F-relaxation, 1: FCF-relaxation (gamma of Algorithm 1) */
    double tol;            /* stop when ||r|| <= tol (x ||r_0|| if tol_relative)         */
    int tol_relative;
    int max_iter;
    int restrict_mode;     /* residual R_s: 0 injection, 1 P^T, 2 diag(P^T 1)^-1 P^T      */
    mg_solver_opts solver;
    int cycle;             /* 0: V-cycle; 1: F-cycle (Sec. 2.1: the coarse system solved by an
                              F-cycle and then a V-cycle on the coarse level)                */
    int nested;            /* initial guess by nested iterations (Sec. 2.1): the coarsest
                              level's problem solved, then level by level interpolated to the
                              C-points, F-relaxed and, below the finest, one V-cycle; 1 with
                              the PWM source, 2 with the sine reference as the source
                              (Sec. 4.1); 0: zero initial guess                              */
    int stop_rule;         /* 0: relative or absolute residual norm (tol, tol_relative); 1: the
                              maximal relative change of the Joule losses at C-points between
                              two iterations <= tol (Sec. 5.1); res_hist then holds that
                              change (the first entry infinite)                            */
    double step_tol_ratio; /* > 0: inexact step solves (no counterpart in the paper): the steps of
                              an iteration are solved to max(solver tolerance, step_tol_ratio x
                              the current relative residual) -- cg_tol, refine_tol and, for
                              Newton steps, newton_tol -- so early iterations, whose iterate
                              is still far from the solution, do not solve to full accuracy; the
                              converged result is unchanged. 0 (default): fixed tolerance    */
} mg_opts;

/* Fill opts with defaults: 2 levels, m = 16, FCF, tol 1e-10 relative,
 * max_iter 50, restrict_mode 2, mg_solver_defaults(), V-cycles, zero initial guess. */
void mg_opts_defaults(mg_opts* opts);

/* FAS-MGRIT (Algorithm 1 with recursive V-cycles) for A u = g, g = (a0, 0, ..., 0)
 * on time level 0 with N steps of T/N on mesh opts->space_level[0].
 * N must be divisible by m[0] * ... * m[L-2].  a0: n doubles; out: (N+1)*n
 * doubles, time-major (device pointers).  Iterate: relax (F or FCF), C-point
 * residual norm, stop test, coarse-grid correction.  Returns MG_EMGRIT_MAXIT if
 * the tolerance was not reached in max_iter iterations and MG_ESTALLED if, with the
 * residual rule, five iterations in a row brought no residual below 0.9 times the
 * smallest one so far (the iterate is then at the accuracy its step solves allow);
 * out holds the last iterate and mg_last_error() the last residual.  Per-column
 * step failures are returned (MG_ECG_MAXIT, MG_ENEWTON) with or without stats. */
mg_status mg_solve(mg_ctx* ctx, int64_t N, double T, const double* a0, double* out,
                   const mg_opts* opts, mg_stats* stats);

/* Estimated device bytes of the work buffers mg_solve(ctx, N, ..., opts) allocates
 * in the context (its level storage, exactly, and the batched-step plans of its
 * relaxation batches; the caller's a0 and out not included) into *bytes.  No
 * device work.  MG_EINVAL for bad options. */
mg_status mg_solve_work_bytes(mg_ctx* ctx, int64_t N, const mg_opts* opts, int64_t* bytes);

/* Frees the context's work buffers: step plans and their CUDA graphs, the solve
 * storage, step work vectors and host staging (all re-created on the next call
 * that needs them).  Meshes, operators, transfers and tuned shapes stay.
 * Synchronises the context's stream. */
mg_status mg_release_work(mg_ctx* ctx);

/* Several independent machine instances at once (the paper has no counterpart):
 * instance i is context ctxs[i] (its own meshes, materials, PWM and stream; the
 * contexts must be distinct and should use distinct streams) solved with N[i],
 * T[i], a0[i], out[i] (device pointers, layouts as mg_solve) by mg_solve with
 * opts[i], or by mg_sequential on opts[i].space_level[0] with opts[i].solver when
 * opts[i].levels == 1.  Each instance is driven by a host worker thread, at most
 * max_threads at a time (0 = one per instance), so the instances' kernels run
 * concurrently on the GPU.
 * work_budget bounds the device memory of the instances' work buffers (the a0 and
 * out of every instance are the caller's and not counted): 0 = no bound (every
 * instance may run at once; work buffers stay allocated afterwards); > 0 = bytes,
 * -1 = the device's free memory at the call less 5 %.  With a bound, instances
 * start in order of decreasing mg_solve_work_bytes, each only while the estimates
 * of the running ones and its own fit the bound (or when none runs), and each
 * instance's work buffers are released (mg_release_work) when it ends; an instance
 * that ran out of device memory next to others is solved again alone at the end.
 * status[i] and stats[i] (either may be NULL) receive each instance's status and
 * statistics; the call returns the worst status and returns when every instance's
 * stream is idle. */
mg_status mg_batch_solve(mg_ctx* const* ctxs, int n, const int64_t* N, const double* T,
                         const double* const* a0, double* const* out, const mg_opts* opts,
                         int max_threads, int64_t work_budget, mg_status* status, mg_stats* stats);

/* Joule losses (Eq. losses, per unit depth) of a trajectory on mesh `level`:
 * losses[i] = d_i^T M_sigma d_i with d_i = (traj[i] - traj[i-1]) / (T/N) for
 * i = 1..N and losses[0] = 0.  traj: (N+1)*n doubles, time-major; losses: N+1
 * doubles (device pointers, caller-owned).  Asynchronous on the stream. */
mg_status mg_joule_losses(mg_ctx* ctx, int level, int64_t N, double T, const double* traj, double* losses);

/* Temporal coarsening plan (Sec. 4.1's heuristic, no GPU work): from measured
 * times ms_list[i] of one batched step of k_list[i] columns, the batch width k*
 * is the smallest one whose throughput (columns per ms) is within 90 % of the
 * best (the counterpart of Sec. 4.1's number of processors); the first
 * coarsening factor m0 is the largest divisor of N (at least 2) with N / m0 >= k*,
 * so that the second grid has about one interval per column of the widest
 * efficient batch; every further level coarsens by coarse_m (0: 2, the factor of
 * Sec. 4.1's worked example; the paper's runs use 4) while N stays divisible and
 * keeps at least 2 intervals and levels < max_levels.  Writes *levels_out and
 * m_out[0 .. levels-2] (the rest 0).  MG_EINVAL if no divisor qualifies or for
 * bad input. */
mg_status mg_choose_levels(const double* k_list, const double* ms_list, int nk, int64_t N, int max_levels,
                           int coarse_m, int* levels_out, int* m_out);

/* Measures batched-step times on mesh fine_level for 16, 32, ..., 1024 columns
 * (at most N/2) and applies mg_choose_levels; then runs 4 MGRIT iterations (from
 * a0 = 0, the other fields of *opts kept) of that plan and of fixed hierarchies
 * (m = 16; 16 x 16; 32 x 16; 8 x 8 x 8 -- those that divide N and fit max_levels)
 * and chooses the one with the least predicted time to opts->tol: measured time
 * per iteration times the iterations that the measured residual reduction per
 * iteration (after the first) needs.  Fills opts->levels, opts->m and
 * opts->space_level (fine_level on the finest time level, coarse_level on the
 * others).  iter_ms (may be NULL) receives the chosen hierarchy's measured time per
 * iteration.  Allocates a trajectory of (N+1) x n doubles; synchronises.  Linear
 * meshes only (MG_EINVAL otherwise). */
mg_status mg_plan_levels(mg_ctx* ctx, int fine_level, int coarse_level, int64_t N, double T, int max_levels,
                         mg_opts* opts, double* iter_ms);

/* As mg_solve / mg_sequential with HOST a0 and out: the call copies a0 to the
 * device, solves, and copies the trajectory back (both copies on the stream). */
mg_status mg_solve_host(mg_ctx* ctx, int64_t N, double T, const double* a0_host,
                        double* out_host, const mg_opts* opts, mg_stats* stats);
mg_status mg_sequential_host(mg_ctx* ctx, int level, int64_t N, double T,
                             const double* a0_host, double* out_host,
                             const mg_solver_opts* opts, mg_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* MGRIT_EM_H */
