"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerances: FP64 forms <= 1e-10 relative L2 per time point (the operators and
single steps much tighter); FP32+FP64-refinement forms <= 1e-6.  The PWM table,
being integer work, is compared bit for bit.
"""

import math

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from synth.model import PwmSpec, machine_model
from oracle import fem, pwm as opwm, stepper
from oracle.problem import MachineProblem, rel_err_per_point

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1912_03106_gb300 import api  # noqa: E402


@pytest.fixture(scope="module")
def meshes():
    return synth.mesh_hierarchy(3)


def make_ctx(meshes, model):
    ctx = api.Context(0)
    ids = api.setup_machine(ctx, meshes, model)
    return ctx, ids


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def lin5k(meshes):
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    ctx, ids = make_ctx(meshes, model)
    yield model, ctx, ids
    ctx.close()


# ------------------------------------------------------------------ set-up parity

@pytest.mark.parametrize("level", [0, 1, 2])
def test_assembly_matches_oracle(meshes, lin5k, level):
    model, ctx, ids = lin5k
    ops = ctx.mg_get_operators(ids[level])
    fe = fem.FEModel(meshes[level], model)
    n = fe.n
    for name, ref in (("K", fe.K), ("M", fe.M)):
        A = sp.csr_matrix((ops[name], ops["col"], ops["rowptr"]), shape=(n, n))
        assert abs(A - ref).max() <= 1e-13 * abs(ref).max(), name
    assert np.abs(ops["F"].T - fe.F).max() <= 1e-15 * max(1.0, np.abs(fe.F).max()) * 10


@pytest.mark.parametrize("N,T,fc,kind", [(256, 5e-3, 5e3, 1), (4096, 20e-3, 20e3, 1), (16384, 20e-3, 20e3, 1),
                                         (4096, 20e-3, 20e3, 0), (1000, 7e-3, 333.3, 1)])
def test_pwm_table_bit_exact(meshes, N, T, fc, kind):
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=fc, carrier=kind))
    ctx, _ = make_ctx(meshes[:1], model)
    got = ctx.mg_pwm_table(N, T)
    want = opwm.sign_table(model.pwm, T, N)
    assert np.array_equal(got, want)
    ctx.close()


# ------------------------------------------------------------------ one batched step

@pytest.mark.parametrize("level,k", [(0, 1), (0, 16), (0, 37), (1, 8), (1, 100), (2, 70)])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("path", [1, 2])
def test_batched_step(meshes, lin5k, level, k, precision, path):
    model, ctx, ids = lin5k
    N, T = 256, 5e-3
    fe = fem.FEModel(meshes[level], model)
    n = fe.n
    rng = np.random.default_rng(level * 1000 + k)
    x_in = 0.01 * rng.standard_normal((n, k))
    dt_mult, i0 = 2, 3
    istride = min(5, (N - i0) // max(1, k - 1))
    signs = opwm.sign_table(model.pwm, T, N)
    phi = stepper.LinearPhi(fe, dt_mult * T / N, stepper.Forcing(fe.F, model.pwm.J0, signs, 1))
    want = np.stack([phi(x_in[:, c], i0 + c * istride) for c in range(k)], axis=1)
    out = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    so = api.solver_opts(precision=precision, cg_tol=1e-14, refine_tol=1e-14, path=path)
    _, st = ctx.mg_step(ids[level], N, T, dev(x_in), out, dt_mult=dt_mult, i0=i0, istride=istride, solver=so)
    got = out.cpu().numpy()
    err = np.linalg.norm(got - want, axis=0) / np.linalg.norm(want, axis=0)
    assert err.max() <= 1e-11, err.max()
    assert st["worst_status"] == "MG_OK"
    assert st["step_solves"] == k


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("nu", [1, 2, 4, 6])
def test_smoothers_give_the_same_step(meshes, lin5k, path, nu):
    """Chebyshev and damped-Jacobi smoothing change only the preconditioner: with
    either, the step on the 18,240-DOF mesh is the oracle's to 1e-11; from two
    sweeps on, Chebyshev needs fewer PCG iterations."""
    model, ctx, ids = lin5k
    N, T, k, i0 = 256, 5e-3, 24, 5
    fe = fem.FEModel(meshes[2], model)
    x_in = 0.01 * np.random.default_rng(nu).standard_normal((fe.n, k))
    signs = opwm.sign_table(model.pwm, T, N)
    phi = stepper.LinearPhi(fe, T / N, stepper.Forcing(fe.F, model.pwm.J0, signs, 1))
    want = np.stack([phi(x_in[:, c], i0 + c) for c in range(k)], axis=1)
    its = []
    for smoother in (0, 1):
        out = torch.zeros((fe.n, k), dtype=torch.float64, device="cuda")
        so = api.solver_opts(cg_tol=1e-14, path=path, smooth=nu, smoother=smoother)
        _, st = ctx.mg_step(ids[2], N, T, dev(x_in), out, i0=i0, istride=1, solver=so)
        err = np.linalg.norm(out.cpu().numpy() - want, axis=0) / np.linalg.norm(want, axis=0)
        assert err.max() <= 1e-11, (smoother, err.max())
        assert st["worst_status"] == "MG_OK"
        its.append(st["cg_iters"])
    if nu >= 2:
        assert its[0] < its[1], its


def test_step_rejects_bad_arguments(meshes, lin5k):
    model, ctx, ids = lin5k
    n = ctx.mg_num_dofs(ids[0])
    x = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_step(ids[0], 16, 1e-3, x, x, i0=15, istride=1)  # time index 18 > N
    assert e.value.status == -1
    with pytest.raises(api.L.MgError):
        ctx.mg_step(99, 16, 1e-3, x, x)
    with pytest.raises(api.L.MgError):
        ctx.mg_step(ids[0], 16, 1e-3, x, x, solver=api.solver_opts(tile=3))
    for bad in (dict(smoother=2), dict(cheb_ratio=1.0), dict(cheb_ratio=-3.0), dict(smooth=9)):
        with pytest.raises(api.L.MgError) as e:
            ctx.mg_step(ids[0], 16, 1e-3, x, x, solver=api.solver_opts(**bad))
        assert e.value.status == -1, bad


@pytest.mark.parametrize("path", [1, 2])
def test_step_iteration_limit_is_reported(meshes, lin5k, path):
    model, ctx, ids = lin5k
    n = ctx.mg_num_dofs(ids[1])
    x_in = dev(0.01 * np.random.default_rng(0).standard_normal((n, 8)))
    out = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    rc, st = ctx.mg_step(ids[1], 256, 5e-3, x_in, out, solver=api.solver_opts(max_cg=3, path=path), allow=(-5,))
    assert rc == -5 and st["worst_status"] == "MG_ECG_MAXIT"


def test_step_paths_agree(meshes, lin5k):
    """Cluster and graph paths compute the same step (different reduction orders)."""
    model, ctx, ids = lin5k
    n = ctx.mg_num_dofs(ids[2])
    x_in = dev(0.01 * np.random.default_rng(4).standard_normal((n, 48)))
    outs = []
    for path in (1, 2):
        out = torch.zeros((n, 48), dtype=torch.float64, device="cuda")
        ctx.mg_step(ids[2], 4096, 20e-3, x_in, out, i0=1, istride=3, solver=api.solver_opts(path=path))
        outs.append(out.cpu().numpy())
    err = np.linalg.norm(outs[0] - outs[1], axis=0) / np.linalg.norm(outs[0], axis=0)
    assert err.max() <= 1e-11


# ------------------------------------------------------------------ sequential stepping

@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-9)])
def test_sequential_matches_oracle(meshes, lin5k, precision, tol):
    model, ctx, ids = lin5k
    N, T = 64, 5e-3 / 4
    ref = MachineProblem(meshes, model, N, T, (0,), ()).sequential()
    n = ref.shape[1]
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty((N + 1, n), dtype=torch.float64, device="cuda")
    ctx.mg_sequential(ids[0], N, T, a0, out, solver=api.solver_opts(precision=precision))
    err = rel_err_per_point(out.cpu().numpy(), ref)
    assert err.max() <= tol, err.max()


# ------------------------------------------------------------------ MGRIT

def run_mgrit(ctx, N, T, n, opts):
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty((N + 1, n), dtype=torch.float64, device="cuda")
    rc, st = ctx.mg_solve(N, T, a0, out, opts, allow=(-7,))
    assert rc == 0, "MGRIT did not reach the tolerance: " + " ".join("%.2e" % h for h in st["res_hist"])
    return out.cpu().numpy(), st


@pytest.mark.parametrize("relax", [0, 1])
def test_two_level_cfg0_matches_sequential_oracle(meshes, lin5k, relax):
    """2-level MGRIT at the 24 x 48 mesh, N = 256, m = 16 (F and FCF), stopped at
    the absolute residual 1e-11, with the residual history of the first
    iterations as the oracle's."""
    model, ctx, ids = lin5k
    N, T = 256, 5e-3
    P = MachineProblem(meshes, model, N, T, (0, 0), (16,))
    ref = P.sequential()
    opts = api.mgrit_opts(levels=2, m=(16,), space_level=(ids[0], ids[0]), relax=relax, tol=1e-11,
                          tol_relative=False)
    got, st = run_mgrit(ctx, N, T, ref.shape[1], opts)
    assert rel_err_per_point(got, ref).max() <= 1e-10
    # iterate parity: the residual history follows the oracle's MGRIT with the same options
    _, hist = P.mgrit(gamma=relax, tol=1e-11, max_iter=st["iters"], tol_relative=False)
    k = min(len(hist), len(st["res_hist"]), 6)
    h_gpu, h_cpu = np.array(st["res_hist"][:k]), np.array(hist[:k])
    assert np.all(np.abs(h_gpu - h_cpu) <= 1e-6 * h_cpu + 1e-9 * h_cpu[0]), (h_gpu, h_cpu)


def test_mgrit_first_iterates_match_oracle(meshes, lin5k):
    """Same options, stopped after 1, 2 and 3 iterations: GPU and oracle iterates agree."""
    model, ctx, ids = lin5k
    N, T = 128, 5e-3 / 2
    P = MachineProblem(meshes, model, N, T, (0, 0), (8,))
    for iters in (1, 2, 3):
        u_cpu, _ = P.mgrit(gamma=1, tol=0.0, max_iter=iters, tol_relative=False)
        opts = api.mgrit_opts(levels=2, m=(8,), space_level=(ids[0], ids[0]), relax=1, tol=0.0,
                              tol_relative=False, max_iter=iters)
        a0 = torch.zeros(u_cpu.shape[1], dtype=torch.float64, device="cuda")
        out = torch.empty(u_cpu.shape, dtype=torch.float64, device="cuda")
        rc, st = ctx.mg_solve(N, T, a0, out, opts, allow=(-7,))
        scale = np.linalg.norm(u_cpu[1:], axis=1).max()
        err = np.linalg.norm(out.cpu().numpy() - u_cpu, axis=1).max() / scale
        assert err <= 1e-9, (iters, err)


@pytest.mark.parametrize("mode", [0, 2])
def test_spatial_coarsening_two_level(meshes, lin5k, mode):
    model, ctx, ids = lin5k
    N, T = 128, 5e-3 / 2
    P = MachineProblem(meshes, model, N, T, (1, 0), (16,), residual_mode=mode)
    ref = P.sequential()
    opts = api.mgrit_opts(levels=2, m=(16,), space_level=(ids[1], ids[0]), relax=1, tol=1e-8, max_iter=40,
                          restrict_mode=mode)
    got, st = run_mgrit(ctx, N, T, ref.shape[1], opts)
    assert rel_err_per_point(got, ref).max() <= 1e-10
    _, hist = P.mgrit(gamma=1, tol=1e-13, max_iter=3)
    h = np.array(st["res_hist"][:3])
    assert np.all(np.abs(h - np.array(hist[:3])) <= 1e-6 * np.array(hist[:3]))


def test_plain_transpose_restriction_follows_oracle(meshes, lin5k):
    """R_s = P^T on the state-space residual over-corrects (row sums of P^T are ~4 per
    refinement); the GPU iteration reproduces the oracle's growing residuals."""
    model, ctx, ids = lin5k
    N, T = 128, 5e-3 / 2
    P = MachineProblem(meshes, model, N, T, (1, 0), (16,), residual_mode=1)
    _, hist = P.mgrit(gamma=1, tol=0.0, max_iter=3, tol_relative=False)
    opts = api.mgrit_opts(levels=2, m=(16,), space_level=(ids[1], ids[0]), relax=1, tol=0.0, tol_relative=False,
                          max_iter=3, restrict_mode=1)
    a0 = torch.zeros(ctx.mg_num_dofs(ids[1]), dtype=torch.float64, device="cuda")
    out = torch.empty((N + 1, a0.numel()), dtype=torch.float64, device="cuda")
    rc, st = ctx.mg_solve(N, T, a0, out, opts, allow=(-7,))
    h = np.array(st["res_hist"][:4])
    assert h[3] > h[1] > h[0]
    assert np.all(np.abs(h - np.array(hist[:4])) <= 1e-6 * np.array(hist[:4]))


def test_three_level_vcycle_with_sc(meshes, lin5k):
    model, ctx, ids = lin5k
    N, T = 256, 5e-3
    P = MachineProblem(meshes, model, N, T, (1, 0, 0), (8, 4))
    ref = P.sequential()
    opts = api.mgrit_opts(levels=3, m=(8, 4), space_level=(ids[1], ids[0], ids[0]), relax=1, tol=1e-8,
                          max_iter=60)
    got, st = run_mgrit(ctx, N, T, ref.shape[1], opts)
    assert rel_err_per_point(got, ref).max() <= 1e-10
    _, hist = P.mgrit(gamma=1, tol=1e-12, max_iter=4)
    h = np.array(st["res_hist"][:4])
    assert np.all(np.abs(h - np.array(hist[:4])) <= 1e-6 * np.array(hist[:4]))


@pytest.mark.parametrize("space,nested", [((0, 0, 0, 0), False), ((1, 0, 0, 0), False), ((1, 1, 0, 0), True),
                                          ((0, 0, 0, 0), True)])
def test_four_level_fcycle_follows_oracle(meshes, lin5k, space, nested):
    """Four-level F-cycles with FCF-relaxation (m = 4, N = 256), without spatial
    coarsening, with direct and with delayed spatial coarsening, zero or
    nested-iteration initial guess: residual history of the first iterations
    as the oracle's, result as sequential stepping."""
    model, ctx, ids = lin5k
    N, T = 256, 5e-3
    P = MachineProblem(meshes, model, N, T, space, (4, 4, 4))
    ref = P.sequential()
    opts = api.mgrit_opts(levels=4, m=(4, 4, 4), space_level=tuple(ids[s] for s in space), relax=1, tol=1e-8,
                          max_iter=40, cycle="F", nested=nested)
    got, st = run_mgrit(ctx, N, T, ref.shape[1], opts)
    assert rel_err_per_point(got, ref).max() <= 1e-9
    _, hist = P.mgrit(gamma=1, tol=0.0, max_iter=3, tol_relative=False, cycle_kind="F", nested=nested)
    k = min(4, len(st["res_hist"]))
    h, hc = np.array(st["res_hist"][:k]), np.array(hist[:k])
    # absolute slack 1e-9 of the first residual: the floor the 1e-13 step solves leave
    assert np.all(np.abs(h - hc) <= 1e-6 * hc + 1e-9 * hc[0]), (h, hc)


def test_nested_guess_alone_matches_oracle(meshes, lin5k):
    """max_iter = 0 with nested iterations: the returned trajectory is the nested
    guess after one relaxation, point by point as the oracle's."""
    model, ctx, ids = lin5k
    N, T = 128, 5e-3 / 2
    P = MachineProblem(meshes, model, N, T, (1, 0, 0), (4, 4))
    u_cpu, _ = P.mgrit(gamma=1, tol=0.0, max_iter=0, tol_relative=False, nested=True)
    opts = api.mgrit_opts(levels=3, m=(4, 4), space_level=(ids[1], ids[0], ids[0]), relax=1, tol=0.0,
                          tol_relative=False, max_iter=0, nested=True)
    a0 = torch.zeros(u_cpu.shape[1], dtype=torch.float64, device="cuda")
    out = torch.empty(u_cpu.shape, dtype=torch.float64, device="cuda")
    ctx.mg_solve(N, T, a0, out, opts, allow=(-7,))
    scale = np.linalg.norm(u_cpu[1:], axis=1).max()
    err = np.linalg.norm(out.cpu().numpy() - u_cpu, axis=1).max() / scale
    assert err <= 1e-10, err


def test_inexact_step_solves_reach_the_same_solution(meshes, lin5k):
    """step_tol_ratio > 0 solves the steps of early iterations loosely; the
    iteration still converges to the sequential solution (tight final stop)."""
    model, ctx, ids = lin5k
    N, T = 256, 5e-3
    ref = MachineProblem(meshes, model, N, T, (1,), ()).sequential()
    opts = api.mgrit_opts(levels=3, m=(8, 4), space_level=(ids[1], ids[0], ids[0]), relax=1, tol=1e-9,
                          max_iter=80, step_tol_ratio=1e-3)
    got, st = run_mgrit(ctx, N, T, ref.shape[1], opts)
    assert rel_err_per_point(got, ref).max() <= 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_mgrit_on_the_graph_path(meshes, lin5k, precision):
    """64 intervals per batched step: the fine level runs on the graph path."""
    model, ctx, ids = lin5k
    N, T = 1024, 5e-3
    ref = MachineProblem(meshes, model, N, T, (0,), ()).sequential()
    so = api.solver_opts(precision=precision)
    opts = api.mgrit_opts(levels=2, m=(16,), space_level=(ids[0], ids[0]), relax=1, tol=1e-9, solver=so)
    got, st = run_mgrit(ctx, N, T, ref.shape[1], opts)
    assert rel_err_per_point(got, ref).max() <= (1e-9 if precision == 0 else 1e-6)


def test_mixed_precision_mgrit(meshes, lin5k):
    model, ctx, ids = lin5k
    N, T = 256, 5e-3
    ref = MachineProblem(meshes, model, N, T, (0,), ()).sequential()
    so = api.solver_opts(precision=1)
    opts = api.mgrit_opts(levels=2, m=(16,), space_level=(ids[0], ids[0]), relax=1, tol=1e-9, solver=so)
    got, st = run_mgrit(ctx, N, T, ref.shape[1], opts)
    assert rel_err_per_point(got, ref).max() <= 1e-6


def test_host_entry_points(meshes, lin5k):
    model, ctx, ids = lin5k
    N, T = 64, 5e-3 / 4
    ref = MachineProblem(meshes, model, N, T, (0,), ()).sequential()
    n = ref.shape[1]
    out = np.empty((N + 1, n))
    opts = api.mgrit_opts(levels=2, m=(8,), space_level=(ids[0], ids[0]), relax=1, tol=1e-9)
    ctx.mg_solve_host(N, T, np.zeros(n), out, opts)
    assert rel_err_per_point(out, ref).max() <= 1e-10
    out2 = np.empty((N + 1, n))
    ctx.mg_sequential_host(ids[0], N, T, np.zeros(n), out2)
    assert rel_err_per_point(out2, ref).max() <= 1e-10


def test_mgrit_rejects_indivisible_N(meshes, lin5k):
    model, ctx, ids = lin5k
    n = ctx.mg_num_dofs(ids[0])
    opts = api.mgrit_opts(levels=2, m=(16,), space_level=(ids[0], ids[0]))
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty((101, n), dtype=torch.float64, device="cuda")
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_solve(100, 1e-3, a0, out, opts)
    assert e.value.status == -1
