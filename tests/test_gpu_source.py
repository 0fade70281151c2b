"""GPU parity of the source options and the loss-based stopping rule: start-up
ramp (Sec. 3.3), nested iterations driven by the sine reference (Sec. 4.1),
Joule losses (Eq. losses) and MGRIT stopped on their relative change (Sec. 5.1)."""

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
    return synth.mesh_hierarchy(2)


def setup(meshes, model, t_ramp=0.0):
    ctx = api.Context(0)
    ids = api.setup_machine(ctx, meshes, model)
    if t_ramp:
        ctx.mg_set_ramp(t_ramp)
    return ctx, ids


def zeros(n):
    return torch.zeros(n, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("nonlinear", [False, True])
def test_ramped_sequential_matches_oracle(meshes, nonlinear):
    model = machine_model(nonlinear=nonlinear, pwm=PwmSpec(J0=3e6 if nonlinear else 1e6, f_carrier=20e3))
    N, T, tr = (32, 32 * 20e-3 / 8192, 2e-4) if nonlinear else (128, 2.5e-3, 1.5e-3)
    ctx, ids = setup(meshes, model, tr)
    P = MachineProblem(meshes, model, N, T, (0,), (), nonlinear=nonlinear, t_ramp=tr)
    ref = P.sequential()
    out = torch.zeros(ref.shape, dtype=torch.float64, device="cuda")
    ctx.mg_sequential(ids[0], N, T, zeros(ref.shape[1]), out)
    assert rel_err_per_point(out.cpu().numpy(), ref).max() <= 1e-10
    ctx.close()


def test_joule_losses_match_oracle(meshes):
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    ctx, ids = setup(meshes, model)
    N, T = 128, 2.5e-3
    P = MachineProblem(meshes, model, N, T, (1,), ())
    u = P.sequential()
    want = P.joule_losses(u)
    losses = torch.empty(N + 1, dtype=torch.float64, device="cuda")
    ctx.mg_joule_losses(ids[1], N, T, torch.as_tensor(u, device="cuda"), losses)
    got = losses.cpu().numpy()
    assert got[0] == 0.0
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    ctx.close()


@pytest.mark.parametrize("space", [(0, 0), (1, 0, 0)])
def test_reference_nested_mgrit_matches_oracle(meshes, space):
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    ctx, ids = setup(meshes, model)
    N, T = 256, 5e-3
    m = (16,) if len(space) == 2 else (8, 4)
    P = MachineProblem(meshes, model, N, T, space, m)
    ref = P.sequential()
    opts = api.mgrit_opts(levels=len(space), m=m, space_level=tuple(ids[s] for s in space), relax=1, tol=1e-8,
                          max_iter=40, nested="reference")
    out = torch.empty(ref.shape, dtype=torch.float64, device="cuda")
    rc, st = ctx.mg_solve(N, T, zeros(ref.shape[1]), out, opts, allow=(-7,))
    assert rc == 0
    assert rel_err_per_point(out.cpu().numpy(), ref).max() <= 1e-9
    _, hist = P.mgrit(gamma=1, tol=0.0, max_iter=3, tol_relative=False, nested="reference")
    k = min(4, len(st["res_hist"]))
    h, hc = np.array(st["res_hist"][:k]), np.array(hist[:k])
    assert np.all(np.abs(h - hc) <= 1e-6 * hc + 1e-9 * hc[0]), (h, hc)
    ctx.close()


def test_joule_stop_rule_matches_oracle(meshes):
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    ctx, ids = setup(meshes, model)
    N, T = 256, 5e-3
    P = MachineProblem(meshes, model, N, T, (0, 0), (16,))
    _, hist = P.mgrit(gamma=1, tol=1e-3, max_iter=20, stop="joule")
    opts = api.mgrit_opts(levels=2, m=(16,), space_level=(ids[0], ids[0]), relax=1, tol=1e-3, max_iter=20,
                          stop="joule")
    out = torch.empty((N + 1, P.n), dtype=torch.float64, device="cuda")
    rc, st = ctx.mg_solve(N, T, zeros(P.n), out, opts, allow=(-7,))
    assert rc == 0
    h = st["res_hist"]
    assert len(h) == len(hist) and h[0] == float("inf")
    assert np.allclose(h[1:], hist[1:], rtol=1e-6, atol=1e-12), (h, hist)
    ctx.close()
