"""Pins of the oracle's backward-Euler propagator and Newton solver (CPU only).

T1: first-order convergence in time on a manufactured semi-discrete solution.
T9: Newton with k1 = 0 equals the linear solve; the Jacobian matches finite
    differences of K(a) a; Newton converges quadratically.
"""

import math

import numpy as np
import pytest

import synth
from synth.model import LAW_BRAUER, Material, MachineModel, PwmSpec, machine_model
from oracle import fem, stepper
from oracle.problem import MachineProblem


@pytest.fixture(scope="module")
def mesh0():
    return synth.annulus_mesh()


def test_backward_euler_first_order(mesh0):
    fe = fem.FEModel(mesh0, machine_model())
    rng = np.random.default_rng(3)
    v = rng.standard_normal(fe.n)
    T, w = 5e-3, 2 * math.pi * 200.0
    Mv, Kv = fe.M @ v, fe.K @ v

    errs = []
    for N in (32, 64, 128, 256):
        dt = T / N

        def forcing(i, dt=dt):
            t = i * dt
            return Mv * w * math.cos(w * t) + Kv * math.sin(w * t)

        phi = stepper.LinearPhi(fe, dt, forcing)
        u = stepper.sequential(phi, N, np.zeros(fe.n))
        errs.append(np.linalg.norm(u[-1] - math.sin(w * T) * v) / np.linalg.norm(v))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(3)]
    assert all(0.93 < q < 1.07 for q in rates), (errs, rates)


def test_sequential_is_forward_block_solve(mesh0):
    # residual of the block-bidiagonal system A u = g vanishes for the sequential solution
    P = MachineProblem([mesh0], machine_model(pwm=PwmSpec(f_carrier=5e3)), 64, 5e-3, (0,), ())
    u = P.sequential()
    phi = P.levels[0].phi
    L, Mdt = phi.L, phi.Mdt
    for i in range(1, 65):
        terms = (L @ u[i], Mdt @ u[i - 1], phi.forcing(i))
        r = terms[0] - terms[1] - terms[2]
        # backward-stable banded Cholesky: residual at rounding level of the largest term
        assert np.linalg.norm(r) <= 1e-11 * max(np.linalg.norm(t) for t in terms)


def _model(k1):
    base = machine_model(nonlinear=True)
    mats = list(base.materials)
    for r, mat in enumerate(mats):
        if mat.law == LAW_BRAUER:
            mats[r] = Material(mat.sigma, mat.nu, LAW_BRAUER, k1, mat.k2, mat.k3)
    return MachineModel(materials=mats, coil_phase=base.coil_phase, pwm=PwmSpec(J0=3e6, f_carrier=5e3))


def test_newton_reduces_to_linear_when_k1_zero(mesh0):
    nl = _model(0.0)
    lin_mats = [Material(m.sigma, m.k3) if m.law == LAW_BRAUER else m for m in nl.materials]
    lin = MachineModel(materials=lin_mats, coil_phase=nl.coil_phase, pwm=nl.pwm)
    Pn = MachineProblem([mesh0], nl, 16, 5e-3, (0,), (), nonlinear=True)
    Pl = MachineProblem([mesh0], lin, 16, 5e-3, (0,), ())
    un, ul = Pn.sequential(), Pl.sequential()
    assert np.abs(un - ul).max() <= 1e-11 * np.abs(ul).max()


def test_jacobian_matches_finite_differences(mesh0):
    # at a saturated state (|B| up to ~2 T) from a few nonlinear steps, random direction
    P = MachineProblem([mesh0], _model(3.8), 64, 5e-3, (0,), (), nonlinear=True)
    fe = P.levels[0].phi.fe
    a = P.sequential()[4]
    d = np.random.default_rng(5).standard_normal(fe.n) * np.abs(a).max()
    eps = 1e-6 * np.linalg.norm(a) / np.linalg.norm(d)
    Fp = fe.stiffness_at(a + eps * d) @ (a + eps * d)
    Fm = fe.stiffness_at(a - eps * d) @ (a - eps * d)
    fd = (Fp - Fm) / (2 * eps)
    Jd = fe.jacobian_at(a) @ d
    assert np.linalg.norm(fd - Jd) <= 1e-6 * np.linalg.norm(Jd)
    # the nonlinearity is active: J differs from K(a)
    assert np.linalg.norm(fe.stiffness_at(a) @ d - Jd) > 1e-3 * np.linalg.norm(Jd)


def test_newton_quadratic_convergence(mesh0):
    P = MachineProblem([mesh0], _model(3.8), 32, 5e-3, (0,), (), nonlinear=True, newton_tol=1e-13)
    phi = P.levels[0].phi
    u = P.sequential()
    # saturation is reached somewhere: |B|^2 large enough that nu grows by > 10 %
    g = phi.fe.grad(u[-1])
    nu, _ = phi.fe.nu_of(np.sum(g * g, axis=1))
    assert nu[phi.fe.law_e == 1].max() > 1.1 * 396.2 + 3.8
    # one step from the last state with a large jump: residual history is quadratic
    phi(u[-1] * 0.0, 32)
    h = np.array(phi.history)
    assert h[-1] <= 1e-10 * h[0]
    # quadratic tail: pairs above the rounding floor h[-1]
    ok = [h[k + 1] <= 10.0 * h[k] ** 2 / h[0] for k in range(len(h) - 1)
          if h[k] < 1e-2 * h[0] and h[k + 1] > 100.0 * h[-1]]
    assert ok and all(ok), h
