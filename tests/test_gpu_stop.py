"""Stopping tests and failure reporting of the GPU path (GPU).

Algorithm 1 stops once the space-time residual falls below a tolerance (Sec. 4.1
uses an absolute one; the library also offers a relative one).  The residual is
r_c = Phi(u_{cm-1}) - u_cm, so it can only reach zero when evaluating Phi on the
converged iterate returns that iterate: every step solve keeps an initial guess
that already solves its system to working precision (its computed residual within
the rounding bound of b - L x).  Then a tolerance far below the accuracy of the
step solves, 1e-12 of the first residual on the two-level problem, is reachable.

Failures are reported as statuses, with or without statistics: step solves that
hit their iteration limit (MG_ECG_MAXIT), non-finite values planted in an input
(MG_ENONFINITE), Newton iteration limits (MG_ENEWTON), and an MGRIT residual that
stops decreasing (MG_ESTALLED).  Every failure is made on the host: the inputs
or options are bad, no device fault is involved.
"""

import ctypes as C

import numpy as np
import pytest

import synth
from synth.model import PwmSpec, machine_model
from oracle.problem import MachineProblem, rel_err_per_point

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1912_03106_gb300 import api  # noqa: E402


@pytest.fixture(scope="module")
def meshes():
    return synth.mesh_hierarchy(3)


@pytest.fixture(scope="module")
def lin(meshes):
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    ctx = api.Context(0)
    ids = api.setup_machine(ctx, meshes, model)
    yield model, ctx, ids
    ctx.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("relax", [0, 1])
@pytest.mark.parametrize("path", [0, 1, 2])
def test_tight_relative_tolerance_is_reached(meshes, lin, relax, path):
    """Two-level MGRIT (N = 64, m = 8) on the 1,104-DOF mesh to 1e-12 of the first
    residual: converges, and every time point is the oracle's sequential solution
    to 1e-10."""
    model, ctx, ids = lin
    N, T = 64, 5e-3 / 4
    ref = MachineProblem(meshes, model, N, T, (0,), ()).sequential()
    n = ref.shape[1]
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty((N + 1, n), dtype=torch.float64, device="cuda")
    opts = api.mgrit_opts(levels=2, m=(8,), space_level=(ids[0], ids[0]), relax=relax, tol=1e-12,
                          solver=api.solver_opts(path=path))
    rc, st = ctx.mg_solve(N, T, a0, out, opts, allow=(-7, -10))
    assert rc == 0, (rc, st["res_hist"])
    # exactness (Sec. 2.1): F-relaxation needs at most N/m iterations, FCF N/(2m)
    assert st["iters"] <= (N // 8 if relax == 0 else N // 16) + 1, st["res_hist"]
    assert rel_err_per_point(out.cpu().numpy(), ref).max() <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("path", [1, 2])
def test_resolving_a_step_from_its_solution_returns_it(meshes, lin, precision, path):
    """A step re-solved with its own solution as the initial guess returns that
    solution bit for bit: the guess passes the working-precision test."""
    model, ctx, ids = lin
    n = ctx.mg_num_dofs(ids[2])
    k = 32
    x_in = dev(0.01 * np.random.default_rng(7).standard_normal((n, k)))
    so = api.solver_opts(precision=precision, path=path)
    out = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    ctx.mg_step(ids[2], 4096, 20e-3, x_in, out, i0=1, istride=3, solver=so)
    again = out.clone()
    _, st = ctx.mg_step(ids[2], 4096, 20e-3, x_in, again, i0=1, istride=3, guess=True, solver=so)
    assert torch.equal(again, out)
    assert st["cg_iters"] == 0


def test_step_failure_is_returned_without_stats(meshes, lin):
    """mg_solve and mg_sequential called through the C ABI with stats = NULL
    return MG_ECG_MAXIT when the step solves hit their iteration limit."""
    model, ctx, ids = lin
    N, T = 64, 5e-3 / 4
    n = ctx.mg_num_dofs(ids[0])
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty((N + 1, n), dtype=torch.float64, device="cuda")
    so = api.solver_opts(max_cg=1)
    opts = api.mgrit_opts(levels=2, m=(8,), space_level=(ids[0], ids[0]), relax=1, tol=1e-9, solver=so)
    rc = ctx.lib.mg_solve(ctx.h, N, T, C.c_void_p(a0.data_ptr()), C.c_void_p(out.data_ptr()), C.byref(opts), None)
    assert rc == -5, rc
    assert b"MG_ECG_MAXIT" in ctx.lib.mg_last_error(ctx.h)
    rc = ctx.lib.mg_sequential(ctx.h, ids[0], N, T, C.c_void_p(a0.data_ptr()), C.c_void_p(out.data_ptr()),
                               C.byref(so), None)
    assert rc == -5, rc


@pytest.mark.parametrize("path", [1, 2])
def test_nan_in_an_input_state_is_reported(meshes, lin, path):
    """A NaN planted (from the host) in one column of a step's input state is
    reported as MG_ENONFINITE; an infinity as well."""
    model, ctx, ids = lin
    n = ctx.mg_num_dofs(ids[1])
    k = 24
    for bad in (float("nan"), float("inf")):
        x = 0.01 * np.random.default_rng(3).standard_normal((n, k))
        x[17, 5] = bad
        out = torch.zeros((n, k), dtype=torch.float64, device="cuda")
        rc, st = ctx.mg_step(ids[1], 256, 5e-3, dev(x), out, i0=1, istride=1, solver=api.solver_opts(path=path),
                             allow=(-11,))
        assert rc == -11 and st["worst_status"] == "MG_ENONFINITE", (bad, rc, st)


def test_nan_in_the_initial_value_is_reported(meshes, lin):
    model, ctx, ids = lin
    N, T = 64, 5e-3 / 4
    n = ctx.mg_num_dofs(ids[0])
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    a0[100] = float("nan")
    out = torch.empty((N + 1, n), dtype=torch.float64, device="cuda")
    opts = api.mgrit_opts(levels=2, m=(8,), space_level=(ids[0], ids[0]), relax=1, tol=1e-9)
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_solve(N, T, a0, out, opts)
    assert e.value.status == -11


def test_stagnation_is_reported(meshes, lin):
    """F-relaxation with spatial coarsening and the plain transpose P^T as residual
    restriction diverges (the oracle's residuals grow 3x per iteration): the
    solve stops with MG_ESTALLED after five iterations without progress instead of
    running to max_iter."""
    model, ctx, ids = lin
    N, T = 128, 5e-3 / 2
    n = ctx.mg_num_dofs(ids[1])
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty((N + 1, n), dtype=torch.float64, device="cuda")
    opts = api.mgrit_opts(levels=2, m=(16,), space_level=(ids[1], ids[0]), relax=0, tol=1e-10, max_iter=40,
                          restrict_mode=1)
    rc, st = ctx.mg_solve(N, T, a0, out, opts, allow=(-10,))
    assert rc == -10 and st["iters"] == 5, (rc, st["iters"], st["res_hist"])
    assert b"stagnated" in ctx.lib.mg_last_error(ctx.h)


def test_newton_iteration_limit_is_reported(meshes):
    """The first step from rest with J0 = 3e6 saturates the iron and needs 20-30
    damped Newton iterations (Sec. 5); with max_newton = 1 it reports MG_ENEWTON."""
    model = machine_model(nonlinear=True, pwm=PwmSpec(J0=3e6, f_carrier=20e3))
    ctx = api.Context(0)
    ids = api.setup_machine(ctx, meshes[:1], model)
    n = ctx.mg_num_dofs(ids[0])
    x = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    rc, st = ctx.mg_step(ids[0], 1024, 5e-3, x, out, i0=1, istride=1, solver=api.solver_opts(max_newton=1),
                         allow=(-6,))
    assert rc == -6 and st["worst_status"] == "MG_ENEWTON"
    ctx.close()
