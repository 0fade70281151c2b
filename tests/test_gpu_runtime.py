"""GPU tests of the runtime around the step kernels: the launch-shape autotuner
and the concurrent solve of many independent machine instances."""

import numpy as np
import pytest

import synth
from synth.model import PwmSpec, machine_model
from synth.workloads import Instance, instances
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


def make_ctx(meshes, model, stream=None):
    ctx = api.Context(0, stream=stream)
    ids = api.setup_machine(ctx, meshes, model)
    return ctx, ids


@pytest.mark.parametrize("level,k", [(2, 256), (0, 16), (0, 1)])
def test_autotune_shape_gives_the_same_step(meshes, level, k):
    """The tuned launch shape solves the step as the oracle does (banded Cholesky),
    to the bar of the other FP64 step tests, and equals the default shape's step."""
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=20e3))
    ctx, ids = make_ctx(meshes, model)
    n = ctx.mg_num_dofs(ids[level])
    xn = 0.01 * np.random.default_rng(k).standard_normal((n, k))
    x = torch.as_tensor(xn, device="cuda")
    ref = torch.zeros_like(x)
    ctx.mg_step(ids[level], 4096, 20e-3, x, ref, i0=1, istride=1 if k > 1 else 0)
    so, ms = ctx.mg_autotune(ids[level], 4096, 20e-3, k)
    assert ms > 0.0
    assert so.path in (1, 2)
    assert so.base_tiles in (0, 1, 2, 4)
    got = torch.zeros_like(x)
    ctx.mg_step(ids[level], 4096, 20e-3, x, got, i0=1, istride=1 if k > 1 else 0, solver=so)
    err = ((got - ref).norm(dim=0) / ref.norm(dim=0)).max().item()
    assert err <= 1e-11, err
    fe = fem.FEModel(meshes[level], model)
    phi = stepper.LinearPhi(fe, 20e-3 / 4096, stepper.Forcing(fe.F, model.pwm.J0,
                                                             opwm.sign_table(model.pwm, 20e-3, 4096), 1))
    g = got.cpu().numpy()
    for c in sorted({0, k // 2, k - 1}):
        want = phi(xn[:, c], 1 + c if k > 1 else 1)
        assert np.linalg.norm(g[:, c] - want) <= 1e-10 * np.linalg.norm(want), c
    # default options now pick the recorded shape: identical to the explicit run
    again = torch.zeros_like(x)
    ctx.mg_step(ids[level], 4096, 20e-3, x, again, i0=1, istride=1 if k > 1 else 0)
    assert torch.equal(again, got)
    ctx.close()


def test_autotune_of_single_steps_first_on_a_fresh_context(meshes):
    """The autotuner's first trials on a new context run the cluster path before any
    solve has set up the context's iteration counters: they must be set up there."""
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=20e3))
    ctx, ids = make_ctx(meshes, model)
    so, ms = ctx.mg_autotune(ids[2], 4096, 20e-3, 1)
    assert ms > 0.0 and so.path in (1, 2)
    ctx.close()


def test_autotune_rejects_nonlinear_mesh(meshes):
    ctx, ids = make_ctx(meshes[:1], machine_model(nonlinear=True, pwm=PwmSpec(J0=3e6, f_carrier=20e3)))
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_autotune(ids[0], 1024, 5e-3, 16)
    assert e.value.status == -1
    ctx.close()


def instance_setup(meshes, inst, stream):
    model = machine_model(nonlinear=inst.nonlinear, pwm=PwmSpec(J0=inst.J0, f_carrier=inst.f_carrier))
    ctx, ids = make_ctx(meshes[:inst.mesh_level + 1], model, stream=stream)
    n = ctx.mg_num_dofs(ids[inst.mesh_level])
    opts = api.mgrit_opts(levels=2, m=(16,), space_level=(ids[inst.mesh_level], ids[inst.mesh_level]), relax=1,
                          tol=1e-8, max_iter=30)
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros((inst.N + 1, n), dtype=torch.float64, device="cuda")
    return ctx, opts, a0, out


def test_batch_solve_equals_one_by_one(meshes):
    """Six uneven instances (meshes l0/l1, N 64/128/256, carriers, J0, one
    nonlinear) solved concurrently give bit-identical trajectories to solving
    each alone."""
    insts = instances(6, seed=3, mesh_levels=(0, 1), Ns=(64, 128, 256), T=2.5e-3, nonlinear_fraction=0.2,
                      nonlinear_levels=(0,))
    streams = [torch.cuda.Stream() for _ in insts]
    setups = [instance_setup(meshes, inst, s) for inst, s in zip(insts, streams)]
    torch.cuda.synchronize()  # inputs were written on torch's stream
    rc, status, stats = api.mg_batch_solve([s[0] for s in setups], [i.N for i in insts], [i.T for i in insts],
                                           [s[2] for s in setups], [s[3] for s in setups], [s[1] for s in setups])
    assert rc == 0, status
    together = [s[3].clone() for s in setups]
    torch.cuda.synchronize()
    for (ctx, opts, a0, out), inst in zip(setups, insts):
        out.zero_()
        torch.cuda.synchronize()
        r, _ = ctx.mg_solve(inst.N, inst.T, a0, out, opts, allow=(-7,))
        assert r == 0
    torch.cuda.synchronize()
    for (ctx, opts, a0, out), tog in zip(setups, together):
        assert torch.equal(out, tog)
        ctx.close()
    assert all(s["iters"] >= 1 for s in stats)


def test_batch_solve_matches_oracle(meshes):
    """Instances solved together by mg_batch_solve, each against the oracle's
    sequential stepping: FP64 and FP32+refinement linear instances on the
    1,104- and 4,512-DOF meshes, a Brauer-law instance with Newton steps."""
    insts = [Instance(0, 64, 2.5e-3, 5e3, 1.0e6, False), Instance(1, 128, 5e-3, 20e3, 2.0e6, False),
             Instance(1, 64, 2.5e-3, 10e3, 0.7e6, False), Instance(0, 32, 1.25e-3, 20e3, 3.0e6, True)]
    precision = [0, 1, 0, 0]
    streams = [torch.cuda.Stream() for _ in insts]
    setups = []
    for inst, s, p in zip(insts, streams, precision):
        ctx, opts, a0, out = instance_setup(meshes, inst, s)
        opts.tol = 1e-10 if inst.nonlinear else 1e-11
        opts.solver.precision = p
        setups.append((ctx, opts, a0, out))
    torch.cuda.synchronize()
    rc, status, stats = api.mg_batch_solve([s[0] for s in setups], [i.N for i in insts], [i.T for i in insts],
                                           [s[2] for s in setups], [s[3] for s in setups], [s[1] for s in setups])
    assert rc == 0, status
    for (ctx, opts, a0, out), inst, p in zip(setups, insts, precision):
        model = machine_model(nonlinear=inst.nonlinear, pwm=PwmSpec(J0=inst.J0, f_carrier=inst.f_carrier))
        ref = MachineProblem(meshes, model, inst.N, inst.T, (inst.mesh_level,), (),
                             nonlinear=inst.nonlinear).sequential()
        err = rel_err_per_point(out.cpu().numpy(), ref).max()
        assert err <= (1e-6 if p else 1e-9 if inst.nonlinear else 1e-10), (inst, err)
        ctx.close()


def test_batch_solve_under_a_work_budget(meshes):
    """With a work budget smaller than any two instances' work buffers the
    scheduler runs the instances one at a time (largest first) and frees each
    one's buffers when it ends: the trajectories are the unbounded call's, bit for
    bit, and the contexts hold no work buffers afterwards."""
    insts = instances(5, seed=7, mesh_levels=(0, 1), Ns=(64, 128, 256), T=2.5e-3, nonlinear_fraction=0.2,
                      nonlinear_levels=(0,))
    setups = [instance_setup(meshes, inst, torch.cuda.Stream()) for inst in insts]
    torch.cuda.synchronize()
    args = ([s[0] for s in setups], [i.N for i in insts], [i.T for i in insts], [s[2] for s in setups],
            [s[3] for s in setups], [s[1] for s in setups])
    rc, status, _ = api.mg_batch_solve(*args)
    assert rc == 0, status
    free = [s[3].clone() for s in setups]
    est = [ctx.mg_solve_work_bytes(inst.N, opts) for (ctx, opts, _, _), inst in zip(setups, insts)]
    assert all(e > 0 for e in est)
    for s in setups:
        s[3].zero_()
    torch.cuda.synchronize()
    rc, status, stats = api.mg_batch_solve(*args, work_budget=min(est) + 1)
    assert rc == 0, status
    torch.cuda.synchronize()
    for s, f in zip(setups, free):
        assert torch.equal(s[3], f)
    for s in setups:
        s[0].close()


def test_work_estimate_covers_a_solve(meshes):
    """mg_solve_work_bytes against the device memory one solve actually takes
    (free memory before and after, with the step operators already built and the
    work buffers released): the estimate is within [0.75, 2] of it, and
    mg_release_work gives the memory back."""
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=20e3))
    ctx, ids = make_ctx(meshes, model)
    N, T = 1024, 5e-3
    n = ctx.mg_num_dofs(ids[2])
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros((N + 1, n), dtype=torch.float64, device="cuda")
    opts = api.mgrit_opts(levels=3, m=(16, 16), space_level=(ids[2], ids[0], ids[0]), relax=1, tol=1e-6)
    ctx.mg_solve(N, T, a0, out, opts)
    ctx.mg_release_work()
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    ctx.mg_solve(N, T, a0, out, opts)
    torch.cuda.synchronize()
    used = before - torch.cuda.mem_get_info()[0]
    est = ctx.mg_solve_work_bytes(N, opts)
    assert used > 0 and 0.75 * used <= est <= 2.0 * used, (used, est)
    ctx.mg_release_work()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= before - (8 << 20)
    ctx.close()


def test_batch_solve_rejects_repeated_context(meshes):
    inst = instances(1, seed=0, mesh_levels=(0,), Ns=(64,), T=2.5e-3, nonlinear_fraction=0.0)[0]
    ctx, opts, a0, out = instance_setup(meshes, inst, torch.cuda.Stream())
    rc, _, _ = api.mg_batch_solve([ctx, ctx], [64, 64], [inst.T, inst.T], [a0, a0], [out, out], [opts, opts])
    assert rc == -1
    ctx.close()


def test_plan_levels_gives_a_converging_hierarchy(meshes):
    """Sec. 4.1's coarsening heuristic on measured step times: the plan divides N,
    and MGRIT with it reaches GPU sequential stepping."""
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=20e3))
    ctx, ids = make_ctx(meshes, model)
    N, T = 4096, 20e-3
    opts, est = ctx.mg_plan_levels(ids[2], ids[0], N, T, max_levels=5,
                                   opts=api.mgrit_opts(tol=1e-4, max_iter=60))
    assert est > 0.0
    prod = 1
    for l in range(opts.levels - 1):
        assert opts.m[l] >= 2
        prod *= opts.m[l]
    assert N % prod == 0 and opts.space_level[0] == ids[2]
    n = ctx.mg_num_dofs(ids[2])
    a0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    seq = torch.empty((N + 1, n), dtype=torch.float64, device="cuda")
    ctx.mg_sequential(ids[2], N, T, a0, seq)
    out = torch.empty_like(seq)
    rc, st = ctx.mg_solve(N, T, a0, out, opts, allow=(-7,))
    assert rc == 0, st["res_hist"]
    err = ((out[1:] - seq[1:]).norm(dim=1) / seq[1:].norm(dim=1)).max().item()
    assert err <= 1e-5, err
    # the oracle's sequential stepping at sampled time points
    fe = fem.FEModel(meshes[2], model)
    phi = stepper.LinearPhi(fe, T / N, stepper.Forcing(fe.F, model.pwm.J0, opwm.sign_table(model.pwm, T, N), 1))
    ref = stepper.sequential(phi, 1024, np.zeros(n))
    got = out[:1025].cpu().numpy()
    assert rel_err_per_point(got, ref).max() <= 1e-5
    print("plan", opts.levels, [opts.m[l] for l in range(opts.levels - 1)], "est ms/iter", est,
          "iters", st["iters"], "solve s", st["t_solve"])
    ctx.close()
