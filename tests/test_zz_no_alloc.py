"""mg_step_static, the batched step that allocates nothing, against mg_step (GPU).

Callers that cannot allocate device memory during a call (stream capture into a
CUDA graph, external memory managers) use mg_step_static; its work vectors live
in the library's fixed static device array.  Its results must equal those of the
allocating mg_step within the step tolerance of the other step tests, on two
calls in a row (the array keeps the previous call's contents).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
from synth.model import PwmSpec, machine_model  # noqa: E402
from oracle import fem, pwm as opwm, stepper  # noqa: E402
from paper_1912_03106_gb300 import api  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    ctx = api.Context(0)
    ids = api.setup_machine(ctx, synth.mesh_hierarchy(2), machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3)))
    yield ctx, ids
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_static_step_matches_allocating_step_twice(setup, precision):
    ctx, ids = setup
    level, N, T, k = ids[1], 256, 5e-3, 24
    n = ctx.mg_num_dofs(level)
    so = api.solver_opts(precision=precision, cg_tol=1e-14, refine_tol=1e-14)
    rng = np.random.default_rng(11 + precision)
    ref = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    x0 = torch.as_tensor(0.01 * rng.standard_normal((n, k)), device="cuda")
    # one regular call builds the step operator and the PWM table
    ctx.mg_step(level, N, T, x0, ref, dt_mult=2, i0=3, istride=5, solver=so)
    for call in range(2):
        x_in = torch.as_tensor(0.01 * rng.standard_normal((n, k)), device="cuda")
        want = torch.zeros((n, k), dtype=torch.float64, device="cuda")
        got = torch.full((n, k), float("nan"), dtype=torch.float64, device="cuda")
        ctx.mg_step(level, N, T, x_in, want, dt_mult=2, i0=3 + call, istride=5, solver=so)
        _, st = ctx.mg_step_static(level, N, T, x_in, got, dt_mult=2, i0=3 + call, istride=5, solver=so)
        w, g = want.cpu().numpy(), got.cpu().numpy()
        err = np.linalg.norm(g - w, axis=0) / np.linalg.norm(w, axis=0)
        assert err.max() <= 1e-11, (call, err.max())
        assert st["worst_status"] == "MG_OK"


def test_static_step_refuses_what_it_cannot_do(setup):
    ctx, ids = setup
    n = ctx.mg_num_dofs(ids[1])
    x = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    # no operator for this dt yet: nothing is built on this path
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_step_static(ids[1], 256, 5e-3, x, x.clone(), dt_mult=7)
    assert e.value.status == -9
    # beyond the static array
    big = torch.zeros((n, 4096), dtype=torch.float64, device="cuda")
    ctx.mg_step(ids[1], 4096, 5e-3, x, x.clone(), dt_mult=1, i0=1, istride=1)
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_step_static(ids[1], 4096, 5e-3, big, big.clone(), dt_mult=1, i0=0, istride=1)
    assert e.value.status == -1 and "static array" in str(e.value)
    # solver options outside their ranges are refused before anything is launched,
    # as by mg_step (9 sweeps exceed the 8 the smoothing weights have room for)
    for bad in (dict(smooth=9), dict(smoother=2), dict(cheb_ratio=1.0), dict(omega=2.0), dict(path=3),
                dict(rows_per_block=8)):
        with pytest.raises(api.L.MgError) as e:
            ctx.mg_step_static(ids[1], 4096, 5e-3, x, x.clone(), dt_mult=1, i0=1, istride=1,
                               solver=api.solver_opts(**bad))
        assert e.value.status == -1, bad


def test_static_step_matches_the_oracle(setup):
    """The allocation-free step against the oracle's backward-Euler step (banded
    Cholesky) directly, on the 4,512-DOF mesh, at the bar of the other FP64 step
    tests."""
    ctx, ids = setup
    level, N, T, k = ids[1], 256, 5e-3, 24
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    fe = fem.FEModel(synth.mesh_hierarchy(2)[1], model)
    x = 0.01 * np.random.default_rng(29).standard_normal((fe.n, k))
    so = api.solver_opts(cg_tol=1e-14)
    x_in = torch.as_tensor(x, device="cuda")
    ctx.mg_step(level, N, T, x_in, torch.zeros_like(x_in), i0=2, istride=3, solver=so)  # builds the operator
    got = torch.full_like(x_in, float("nan"))
    ctx.mg_step_static(level, N, T, x_in, got, i0=2, istride=3, solver=so)
    phi = stepper.LinearPhi(fe, T / N, stepper.Forcing(fe.F, model.pwm.J0, opwm.sign_table(model.pwm, T, N), 1))
    g = got.cpu().numpy()
    for c in range(k):
        want = phi(x[:, c], 2 + 3 * c)
        assert np.linalg.norm(g[:, c] - want) <= 1e-11 * np.linalg.norm(want), c
