"""Parity at the workloads' full sizes, in the launch configurations the solver
and bench.py use, on outputs the oracle can compute one by one.

cfg1: 18,240 DOFs, N = 4,096, 3-level FCF MGRIT with coarse levels on the 1,104-DOF
mesh (the bench's solve), and its level-0 batched step of 256 columns.
cfg2: 73,344 DOFs, N = 16,384, FP32+refinement: the level-0 batched step of 1,024
columns, and a 256-step prefix of the time grid through 3-level MGRIT with the
workload's delayed spatial coarsening.
cfg3: 18,240 DOFs with the Brauer law, N = 8,192: the level-0 batched Newton step
of 512 columns.
Sampled columns / time points are compared with the oracle (banded Cholesky /
Newton with banded Cholesky).  Bars: FP64 forms 1e-10 relative L2, FP32+refinement
1e-6 (its steps are refined to 1e-13, so they land far below the bar).
"""

import numpy as np
import pytest

import synth
from synth.model import PwmSpec, machine_model
from synth.workloads import workload
from oracle import fem, pwm as opwm, stepper
from oracle.problem import rel_err_per_point

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1912_03106_gb300 import api  # noqa: E402


@pytest.fixture(scope="module")
def meshes():
    return synth.mesh_hierarchy(4)


def setup(meshes, model, levels):
    ctx = api.Context(0)
    ids = api.setup_machine(ctx, meshes[:levels], model)
    return ctx, ids


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def sampled_step_check(ctx, ids, meshes, model, w, level, k, precision, phi_cls, tol, cols, x_in=None):
    fe = fem.FEModel(meshes[level], model)
    n = fe.n
    if x_in is None:
        x_in = 0.01 * np.random.default_rng(level * 7 + k).standard_normal((n, k))
    out = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    so = api.solver_opts(precision=precision)
    _, st = ctx.mg_step(ids[level], w.N, w.T, dev(x_in), out, i0=1, istride=1, solver=so)
    got = out.cpu().numpy()
    signs = opwm.sign_table(model.pwm, w.T, w.N)
    phi = phi_cls(fe, w.T / w.N, stepper.Forcing(fe.F, model.pwm.J0, signs, 1))
    for c in cols:
        want = phi(x_in[:, c], 1 + c)
        err = np.linalg.norm(got[:, c] - want) / np.linalg.norm(want)
        assert err <= tol, (c, err)
    assert st["worst_status"] == "MG_OK"
    return st


def test_cfg1_level0_step_256_columns(meshes):
    w = workload("cfg1_linear_l2_N4096")
    model = machine_model(pwm=PwmSpec(J0=w.J0, f_carrier=w.f_carrier))
    ctx, ids = setup(meshes, model, 3)
    sampled_step_check(ctx, ids, meshes, model, w, 2, w.N // w.m[0], 0, stepper.LinearPhi, 1e-10,
                       cols=(0, 1, 77, 128, 254, 255))
    ctx.close()


def test_cfg1_mgrit_full_size_matches_oracle_samples(meshes):
    """The bench's solve (3-level FCF, m = 16, coarse levels on the 1,104-DOF mesh)
    to 3e-8 relative residual; time points 1, 17, 1024, 2049 and 4096, and then all
    of them, against the oracle's sequential stepping.  With spatial coarsening the
    residual falls about 0.6x per iteration down to a floor near 7e-9 relative (set
    by the 1e-13 tolerance of each step solve), so the stop sits above that floor."""
    w = workload("cfg1_linear_l2_N4096")
    model = machine_model(pwm=PwmSpec(J0=w.J0, f_carrier=w.f_carrier))
    ctx, ids = setup(meshes, model, 3)
    n = ctx.mg_num_dofs(ids[2])
    out = torch.empty((w.N + 1, n), dtype=torch.float64, device="cuda")
    opts = api.mgrit_opts(levels=3, m=(16, 16), space_level=(ids[2], ids[0], ids[0]), relax=1, tol=3e-8,
                          max_iter=100)
    rc, st = ctx.mg_solve(w.N, w.T, torch.zeros(n, dtype=torch.float64, device="cuda"), out, opts, allow=(-7,))
    assert rc == 0, " ".join("%.2e" % h for h in st["res_hist"])
    got = out.cpu().numpy()
    fe = fem.FEModel(meshes[2], model)
    signs = opwm.sign_table(model.pwm, w.T, w.N)
    phi = stepper.LinearPhi(fe, w.T / w.N, stepper.Forcing(fe.F, model.pwm.J0, signs, 1))
    ref = stepper.sequential(phi, w.N, np.zeros(n))
    for i in (1, 17, 1024, 2049, 4096):
        err = np.linalg.norm(got[i] - ref[i]) / np.linalg.norm(ref[i])
        assert err <= 1e-10, (i, err)
    assert rel_err_per_point(got, ref).max() <= 1e-10
    ctx.close()


def test_cfg2_level0_step_1024_columns_mixed(meshes):
    w = workload("cfg2_mixed_l3_N16384")
    model = machine_model(pwm=PwmSpec(J0=w.J0, f_carrier=w.f_carrier))
    ctx, ids = setup(meshes, model, 4)
    sampled_step_check(ctx, ids, meshes, model, w, 3, w.N // w.m[0], 1, stepper.LinearPhi, 1e-6,
                       cols=(0, 511, 1023))
    ctx.close()


def test_cfg2_prefix_mgrit_mixed(meshes):
    """The first 256 steps of the cfg2 time grid (dt = 20 ms / 16,384) through
    3-level FCF MGRIT (m = 16, the workload's delayed spatial coarsening: level 1 on
    the 73,344-DOF mesh, the coarsest level on the 18,240-DOF mesh) in the
    FP32+refinement form: every time point within 1e-6 of the oracle."""
    w = workload("cfg2_mixed_l3_N16384")
    model = machine_model(pwm=PwmSpec(J0=w.J0, f_carrier=w.f_carrier))
    ctx, ids = setup(meshes, model, 4)
    Np = 256
    Tp = w.T * Np / w.N
    n = ctx.mg_num_dofs(ids[3])
    out = torch.empty((Np + 1, n), dtype=torch.float64, device="cuda")
    opts = api.mgrit_opts(levels=3, m=(16, 16), space_level=tuple(ids[s] for s in w.space_levels), relax=1,
                          tol=1e-6, max_iter=100, solver=api.solver_opts(precision=1))
    rc, st = ctx.mg_solve(Np, Tp, torch.zeros(n, dtype=torch.float64, device="cuda"), out, opts, allow=(-7,))
    assert rc == 0, " ".join("%.2e" % h for h in st["res_hist"])
    fe = fem.FEModel(meshes[3], model)
    signs = opwm.sign_table(model.pwm, Tp, Np)
    phi = stepper.LinearPhi(fe, Tp / Np, stepper.Forcing(fe.F, model.pwm.J0, signs, 1))
    ref = stepper.sequential(phi, Np, np.zeros(n))
    assert rel_err_per_point(out.cpu().numpy(), ref).max() <= 1e-6
    ctx.close()


def test_cfg3_level0_newton_step_512_columns(meshes):
    """Batched Newton step of 512 columns from rest at times 1..512 of the cfg3
    grid; two columns (the first step and one mid-grid) against the oracle."""
    w = workload("cfg3_nonlinear_l2_N8192")
    model = machine_model(nonlinear=True, pwm=PwmSpec(J0=w.J0, f_carrier=w.f_carrier))
    ctx, ids = setup(meshes, model, 3)
    n = ctx.mg_num_dofs(ids[2])
    k = w.N // w.m[0]
    st = sampled_step_check(ctx, ids, meshes, model, w, 2, k, 0, stepper.NewtonPhi, 1e-10, cols=(0, 300),
                            x_in=np.zeros((n, k)))
    assert st["newton_iters"] >= k
    ctx.close()
