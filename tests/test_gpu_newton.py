"""GPU parity of the nonlinear (Brauer-law) steps against the CPU oracle.

Sec. 5: with the Brauer law each backward-Euler step is a nonlinear system
solved by damped Newton.  The oracle solves every Newton correction with a
banded Cholesky factorisation; the GPU path with multigrid-preconditioned PCG
on per-column Jacobians.  Both stop once the full correction is below 1e-8 of
the iterate, after which the iterate is accurate to rounding (quadratic
convergence), so the results agree far below the Newton tolerance: the bar is
1e-10 relative L2 per column or time point, as for the linear FP64 path.
"""

import numpy as np
import pytest

import synth
from synth.model import PwmSpec, machine_model
from oracle import fem, pwm as opwm, stepper
from oracle.problem import MachineProblem, rel_err_per_point

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1912_03106_gb300 import api  # noqa: E402

N, T = 1024, 5e-3  # dt = 4.9 us


@pytest.fixture(scope="module")
def meshes():
    return synth.mesh_hierarchy(3)


@pytest.fixture(scope="module")
def nl(meshes):
    # J0 = 3e6 drives the stator iron into saturation (|B| up to 2.25 T)
    model = machine_model(nonlinear=True, pwm=PwmSpec(J0=3e6, f_carrier=20e3))
    ctx = api.Context(0)
    ids = api.setup_machine(ctx, meshes, model)
    yield model, ctx, ids
    ctx.close()


_traj = {}


def oracle_run(meshes, model, level, steps):
    """Sequential oracle states u_0 .. u_steps and Newton iterations per step."""
    key = (level, steps)
    if key not in _traj:
        fe = fem.FEModel(meshes[level], model)
        signs = opwm.sign_table(model.pwm, T, N)
        phi = stepper.NewtonPhi(fe, T / N, stepper.Forcing(fe.F, model.pwm.J0, signs, 1))
        u = [np.zeros(fe.n)]
        its = []
        for i in range(1, steps + 1):
            u.append(phi(u[-1], i))
            its.append(phi.last_iters)
        _traj[key] = (np.array(u), its)
    return _traj[key]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("level,k", [(0, 1), (0, 12), (0, 40), (1, 20), (2, 16)])
def test_newton_step_matches_oracle(meshes, nl, level, k):
    """Columns c = 0..k-1 step from the oracle's u_c at time c+1: the results are
    the oracle's u_{c+1}, including the first step from rest (the iron saturates
    within it and the step needs 20-30 damped iterations)."""
    model, ctx, ids = nl
    u, its = oracle_run(meshes, model, level, k)
    n = u.shape[1]
    out = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    _, st = ctx.mg_step(ids[level], N, T, dev(u[:k].T), out, i0=1, istride=1)
    got = out.cpu().numpy()
    want = u[1:k + 1].T
    err = np.linalg.norm(got - want, axis=0) / np.linalg.norm(want, axis=0)
    assert err.max() <= 1e-10, err.max()
    assert st["worst_status"] == "MG_OK"
    assert st["step_solves"] == k
    # same damped-Newton decisions: iteration totals agree up to a borderline stop per column
    assert abs(st["newton_iters"] - sum(its)) <= k, (st["newton_iters"], sum(its))


def test_newton_smoothers_give_the_same_step(meshes, nl):
    """Chebyshev smoothing of the per-column Jacobians (interval from the device-side
    Gershgorin bound of every Jacobian) and damped Jacobi solve the same Newton
    corrections: both steps are the oracle's to 1e-10, and Chebyshev needs fewer
    PCG iterations.  Switching the smoother on one context also rebuilds the
    correction's cached graph."""
    model, ctx, ids = nl
    k = 20
    u, its = oracle_run(meshes, model, 1, k)
    n = u.shape[1]
    want = u[1:k + 1].T
    cg = {}
    for smoother in (1, 0, 1):
        out = torch.zeros((n, k), dtype=torch.float64, device="cuda")
        _, st = ctx.mg_step(ids[1], N, T, dev(u[:k].T), out, i0=1, istride=1,
                            solver=api.solver_opts(smoother=smoother))
        err = np.linalg.norm(out.cpu().numpy() - want, axis=0) / np.linalg.norm(want, axis=0)
        assert err.max() <= 1e-10, (smoother, err.max())
        assert st["worst_status"] == "MG_OK"
        cg.setdefault(smoother, []).append(st["cg_iters"])
    assert cg[1][0] == cg[1][1], cg  # the rebuilt Jacobi graph repeats the first run
    assert cg[0][0] < cg[1][0], cg


def test_newton_step_from_a_converged_guess(meshes, nl):
    """Started at the solution, every column stops after one (negligible) correction."""
    model, ctx, ids = nl
    k = 12
    u, _ = oracle_run(meshes, model, 0, k)
    n = u.shape[1]
    out = dev(u[1:k + 1].T)
    _, st = ctx.mg_step(ids[0], N, T, dev(u[:k].T), out, i0=1, istride=1, guess=True)
    err = np.linalg.norm(out.cpu().numpy() - u[1:k + 1].T, axis=0) / np.linalg.norm(u[1:k + 1], axis=1)
    assert err.max() <= 1e-10
    assert st["newton_iters"] == k


def test_newton_with_k1_zero_is_the_linear_step(meshes):
    """k1 = 0 makes the Brauer law nu = k3: the Newton step must reproduce the
    linear step with nu = k3 in those regions (T9 of the oracle, on the GPU)."""
    base = machine_model(nonlinear=True, pwm=PwmSpec(J0=3e6, f_carrier=20e3))
    nl_mats = [type(m)(m.sigma, m.nu, m.law, 0.0, m.k2, m.k3) for m in base.materials]
    lin_mats = [type(m)(m.sigma, m.k3 if m.law == 1 else m.nu) for m in base.materials]
    k = 16
    outs = []
    for mats in (nl_mats, lin_mats):
        model = type(base)(materials=mats, coil_phase=base.coil_phase, pwm=base.pwm)
        ctx = api.Context(0)
        ids = api.setup_machine(ctx, meshes[:2], model)
        n = ctx.mg_num_dofs(ids[1])
        x = 0.01 * np.random.default_rng(3).standard_normal((n, k))
        out = torch.zeros((n, k), dtype=torch.float64, device="cuda")
        ctx.mg_step(ids[1], N, T, dev(x), out, i0=5, istride=3)
        outs.append(out.cpu().numpy())
        ctx.close()
    err = np.linalg.norm(outs[0] - outs[1], axis=0) / np.linalg.norm(outs[1], axis=0)
    assert err.max() <= 1e-11, err.max()


def test_nonlinear_sequential_matches_oracle(meshes, nl):
    model, ctx, ids = nl
    steps = 24
    u, _ = oracle_run(meshes, model, 0, steps)
    n = u.shape[1]
    out = torch.zeros((steps + 1, n), dtype=torch.float64, device="cuda")
    # the first `steps` steps of the N-step grid: T scaled so dt stays T / N
    ctx.mg_sequential(ids[0], steps, T * steps / N, torch.zeros(n, dtype=torch.float64, device="cuda"), out)
    err = rel_err_per_point(out.cpu().numpy(), u)
    assert err.max() <= 1e-10, err.max()


def test_nonlinear_mgrit_matches_oracle_iterates(meshes, nl):
    """Two-level FAS-MGRIT, FCF, on the 1,104-DOF mesh: the residual history of
    every iteration agrees with the oracle's, and the result with sequential
    stepping."""
    model, ctx, ids = nl
    Nm, m = 64, 8
    Tm = Nm * T / N
    P = MachineProblem(meshes[:1], model, Nm, Tm, (0, 0), (m,), nonlinear=True)
    seq = P.sequential()
    n = seq.shape[1]
    out = torch.zeros((Nm + 1, n), dtype=torch.float64, device="cuda")
    opts = api.mgrit_opts(levels=2, m=(m,), space_level=(ids[0], ids[0]), relax=1, tol=1e-9, max_iter=30)
    rc, st = ctx.mg_solve(Nm, Tm, torch.zeros(n, dtype=torch.float64, device="cuda"), out, opts, allow=(-7,))
    assert rc == 0, st["res_hist"]
    assert rel_err_per_point(out.cpu().numpy(), seq).max() <= 1e-9
    _, hist = P.mgrit(gamma=1, tol=1e-9, max_iter=st["iters"])
    h_gpu, h_cpu = np.array(st["res_hist"]), np.array(hist)
    assert len(h_gpu) == len(h_cpu), (h_gpu, h_cpu)
    assert np.all(np.abs(h_gpu - h_cpu) <= 1e-6 * h_cpu + 1e-9 * h_cpu[0]), (h_gpu, h_cpu)
    assert st["newton_iters"] > 0


def test_nonlinear_mgrit_with_spatial_coarsening_follows_oracle(meshes, nl):
    """Two-level FAS-MGRIT, FCF, with spatial coarsening (Sec. 2.2) under the
    Brauer law: fine level on the 4,512-DOF mesh, coarse level on the 1,104-DOF
    mesh (the coarse Newton steps evaluate the law on the coarse mesh).  The
    iterates after one and two iterations are the oracle's (the residual history
    too), and the iteration converges to the oracle's sequential Newton stepping."""
    model, ctx, ids = nl
    Nm, m = 16, 4
    Tm = Nm * T / N
    P = MachineProblem(meshes[:2], model, Nm, Tm, (1, 0), (m,), nonlinear=True)
    seq = MachineProblem(meshes[:2], model, Nm, Tm, (1,), (), nonlinear=True).sequential()
    n = seq.shape[1]
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    for iters in (1, 2):
        u_cpu, hist = P.mgrit(gamma=1, tol=0.0, max_iter=iters, tol_relative=False)
        out = torch.zeros((Nm + 1, n), dtype=torch.float64, device="cuda")
        opts = api.mgrit_opts(levels=2, m=(m,), space_level=(ids[1], ids[0]), relax=1, tol=0.0,
                              tol_relative=False, max_iter=iters)
        rc, st = ctx.mg_solve(Nm, Tm, a0, out, opts, allow=(-7,))
        scale = np.linalg.norm(u_cpu[1:], axis=1).max()
        err = np.linalg.norm(out.cpu().numpy() - u_cpu, axis=1).max() / scale
        assert err <= 1e-9, (iters, err)
        h_gpu, h_cpu = np.array(st["res_hist"]), np.array(hist)
        assert np.all(np.abs(h_gpu - h_cpu) <= 1e-6 * h_cpu + 1e-9 * h_cpu[0]), (h_gpu, h_cpu)
    out = torch.zeros((Nm + 1, n), dtype=torch.float64, device="cuda")
    opts = api.mgrit_opts(levels=2, m=(m,), space_level=(ids[1], ids[0]), relax=1, tol=1e-9, max_iter=40)
    rc, st = ctx.mg_solve(Nm, Tm, a0, out, opts, allow=(-7,))
    assert rc == 0, st["res_hist"]
    assert rel_err_per_point(out.cpu().numpy(), seq).max() <= 1e-8


def test_static_step_rejects_nonlinear_mesh(meshes, nl):
    model, ctx, ids = nl
    n = ctx.mg_num_dofs(ids[0])
    x = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    ctx.mg_step(ids[0], N, T, x, x.clone(), i0=1, istride=1)
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_step_static(ids[0], N, T, x, x.clone(), i0=1, istride=1)
    assert e.value.status == -1
