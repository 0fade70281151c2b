"""Kernel variants of the graph path (GPU): halo-fused multigrid kernels and the
cores of the dense base solve.

With `halo_fusion` 2 the V-cycle runs two consecutive smoothing sweeps per launch
(the first sweep's residual formed in shared memory on a halo of the operator's
bandwidth, the second gathered from there) and the prolongation together with the
residual update (the prolongated correction likewise kept in shared memory); with 3
the sweeps' input is staged in shared memory as well.  The kernels do the
arithmetic of the single-phase kernels in the same order, so a batched step with
`halo_fusion` 2 or 3 must give the step with 1: the same PCG
iteration counts and the same result (to rounding), and both the oracle's exact
step solve (banded Cholesky of L = M/dt + K) to the bar of the other FP64 step
tests.  Cases: several 16-column tiles with a ragged last one, 8- and 16-column
block shapes (the library picks by mesh and batch size), both precision forms,
odd and even sweep counts (pairs only, or pairs and single sweeps).

The dense base solve x = A^-1 r runs on the CUDA cores (FP32 FMA) or on the
tensor cores (3xTF32 mma.sync); both are FP32-accurate preconditioner pieces,
so both steps meet the oracle's bar; 1, 2 and 4 tiles per block, ragged tiles.

Steps of the FP64 form with cg_tol >= 1e-8 form the operator products of the
Krylov update in double-float FP32 arithmetic; their true residual, computed on the
CPU with the oracle's matrices, must meet the requested tolerance.
"""

import numpy as np
import pytest

import synth
from synth.model import PwmSpec, machine_model
from oracle import fem, pwm as opwm, stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1912_03106_gb300 import api  # noqa: E402

N, T = 4096, 20e-3


@pytest.fixture(scope="module")
def setup():
    meshes = synth.mesh_hierarchy(3)
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=20e3))
    ctx = api.Context(0)
    ids = api.setup_machine(ctx, meshes, model)
    yield meshes, model, ctx, ids
    ctx.close()


def oracle_step(meshes, model, level, x, t):
    fe = fem.FEModel(meshes[level], model)
    phi = stepper.LinearPhi(fe, T / N, stepper.Forcing(fe.F, model.pwm.J0, opwm.sign_table(model.pwm, T, N), 1))
    return phi(x, t)


@pytest.mark.parametrize("level,k,precision,smooth", [
    (2, 256, 0, 5),   # the dominant launch of the MGRIT solves
    (2, 40, 0, 5),    # three tiles, the last one half full
    (1, 40, 1, 4),    # FP32+refinement, even sweep count
    (2, 100, 1, 3),
    (1, 256, 0, 2),
])
def test_halo_fused_kernels_give_the_same_step(setup, level, k, precision, smooth):
    meshes, model, ctx, ids = setup
    n = ctx.mg_num_dofs(ids[level])
    xn = 0.01 * np.random.default_rng(1000 * level + k).standard_normal((n, k))
    x = torch.as_tensor(xn, device="cuda")
    out = {}
    its = {}
    for hf in (1, 2, 3):
        so = api.solver_opts(path=2, precision=precision, smooth=smooth, halo_fusion=hf)
        y = torch.zeros_like(x)
        _, st = ctx.mg_step(ids[level], N, T, x, y, i0=1, istride=1, solver=so)
        out[hf], its[hf] = y, st["cg_iters"]
    for hf in (2, 3):
        assert abs(its[1] - its[hf]) <= k // 16, its
        diff = ((out[hf] - out[1]).norm(dim=0) / out[1].norm(dim=0)).max().item()
        assert diff <= 1e-11, (hf, diff)
    g = out[3].cpu().numpy()
    for c in sorted({0, k // 2, k - 1}):
        want = oracle_step(meshes, model, level, xn[:, c], 1 + c)
        assert np.linalg.norm(g[:, c] - want) <= 1e-10 * np.linalg.norm(want), c


def test_halo_fusion_is_validated(setup):
    meshes, model, ctx, ids = setup
    n = ctx.mg_num_dofs(ids[0])
    x = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_step(ids[0], N, T, x, y, solver=api.solver_opts(halo_fusion=4))
    assert e.value.status == -1


@pytest.mark.parametrize("level,k,tiles", [(2, 256, 2), (2, 40, 4), (1, 24, 1), (2, 100, 0)])
def test_base_solve_on_cuda_and_tensor_cores(setup, level, k, tiles):
    meshes, model, ctx, ids = setup
    n = ctx.mg_num_dofs(ids[level])
    xn = 0.01 * np.random.default_rng(77 + k).standard_normal((n, k))
    x = torch.as_tensor(xn, device="cuda")
    out, its = {}, {}
    for bc in (1, 2):
        so = api.solver_opts(path=2, base_cores=bc, base_tiles=tiles)
        y = torch.zeros_like(x)
        _, st = ctx.mg_step(ids[level], N, T, x, y, i0=1, istride=1, solver=so)
        out[bc], its[bc] = y, st["cg_iters"]
    assert abs(its[1] - its[2]) <= max(2, k // 8), its
    for c in sorted({0, k // 2, k - 1}):
        want = oracle_step(meshes, model, level, xn[:, c], 1 + c)
        for bc in (1, 2):
            got = out[bc][:, c].cpu().numpy()
            assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want), (bc, c)


@pytest.mark.parametrize("level,k,tol", [(2, 256, 1e-8), (2, 40, 1e-6), (1, 64, 3e-5)])
def test_double_float_products_meet_the_tolerance(setup, level, k, tol):
    """Per column ||b - L x|| <= 1.01 tol ||b|| with b = (M/dt) x_prev + f(t_i) and
    L = M/dt + K from the oracle's FE matrices, and the step agrees with the
    oracle's exact solve to the accuracy the tolerance allows."""
    meshes, model, ctx, ids = setup
    n = ctx.mg_num_dofs(ids[level])
    xn = 0.01 * np.random.default_rng(500 + k).standard_normal((n, k))
    x = torch.as_tensor(xn, device="cuda")
    y = torch.zeros_like(x)
    _, st = ctx.mg_step(ids[level], N, T, x, y, i0=1, istride=1, solver=api.solver_opts(path=2, cg_tol=tol))
    assert st["worst_status"] in (0, "MG_OK"), st
    fe = fem.FEModel(meshes[level], model)
    forcing = stepper.Forcing(fe.F, model.pwm.J0, opwm.sign_table(model.pwm, T, N), 1)
    phi = stepper.LinearPhi(fe, T / N, forcing)
    g = y.cpu().numpy()
    for c in sorted({0, 1, k // 2, k - 1}):
        b = phi.Mdt @ xn[:, c] + forcing(1 + c)
        r = b - phi.L @ g[:, c]
        assert np.linalg.norm(r) <= 1.01 * tol * np.linalg.norm(b), (c, np.linalg.norm(r) / np.linalg.norm(b))
