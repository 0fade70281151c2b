"""Pins of the oracle's FAS-MGRIT (Algorithm 1), CPU only.

T2: one level, or m = 1 with the same coarse propagator, reproduces sequential stepping.
T3: exactness (Sec. 2.1): without spatial coarsening F-relaxation is exact after
    N/m and FCF after N/(2m) iterations; the exact front advances 1 (F) or 2
    (FCF) C-points per iteration.
T4: one two-level iteration on u' = lambda u maps the C-point error e to E e with
    E_F[i,j] = (phi^m - phi_c) phi_c^(i-j-1) (i > j),
    E_FCF[i,j] = phi^m (phi^m - phi_c) phi_c^(i-j-2) (i >= j+2)
    (ideal interpolation makes the Galerkin coarse operator the Schur complement
    with phi^m on its sub-diagonal, Sec. 2.1; the coarse operator re-discretises
    with phi_c).
    Also: two-level MGRIT with F-relaxation is Parareal (Sec. 2.1), checked against
    an independent Parareal recursion.
T10: with spatial coarsening the iteration converges to the same sequential solution.
"""

import numpy as np
import pytest

import synth
from synth.model import PwmSpec, machine_model
from oracle import mgrit, scalar
from oracle.problem import MachineProblem, rel_err_per_point


@pytest.fixture(scope="module")
def meshes():
    return synth.mesh_hierarchy(2)


@pytest.fixture(scope="module")
def model():
    return machine_model(pwm=PwmSpec(f_carrier=5e3))


def closed_form(lam, dt, m, NT, gamma):
    phi = 1.0 / (1.0 - lam * dt)
    phic = 1.0 / (1.0 - lam * m * dt)
    E = np.zeros((NT + 1, NT + 1))
    for i in range(NT + 1):
        for j in range(1, NT + 1):
            if gamma == 0 and i > j:
                E[i, j] = (phi**m - phic) * phic ** (i - j - 1)
            if gamma == 1 and i >= j + 2:
                E[i, j] = phi**m * (phi**m - phic) * phic ** (i - j - 2)
    return E


@pytest.mark.parametrize("lam", [-1.0, -100.0, -1e4])
@pytest.mark.parametrize("m", [4, 16])
@pytest.mark.parametrize("NT", [6, 9])
@pytest.mark.parametrize("gamma", [0, 1])
def test_two_level_error_closed_form(lam, m, NT, gamma):
    dt = 1e-3
    levels = scalar.two_level(lam, dt, m, NT)
    rng = np.random.default_rng(m * 100 + NT)
    e = np.r_[0.0, rng.standard_normal(NT)]
    out = scalar.cpoint_error_after_one_iteration(levels, e, gamma)
    E = closed_form(lam, dt, m, NT, gamma)
    assert np.abs(out - E @ e).max() <= 1e-13 * np.abs(e).max()


def test_closed_form_catches_wrong_coarse_propagator():
    # a planted mistake (coarse step dt instead of m dt) must fail the pin
    lam, dt, m, NT = -100.0, 1e-3, 4, 6
    levels = scalar.two_level(lam, dt, m, NT)
    levels[1].phi = scalar.ScalarPhi(lam, dt)
    e = np.r_[0.0, np.ones(NT)]
    out = scalar.cpoint_error_after_one_iteration(levels, e, 0)
    assert np.abs(out - closed_form(lam, dt, m, NT, 0) @ e).max() > 1e-3


def test_parareal_equivalence():
    lam, dt, m, NT = -30.0, 2e-3, 5, 8
    levels = scalar.two_level(lam, dt, m, NT)
    phi, phic = levels[0].phi.phi, levels[1].phi.phi
    rng = np.random.default_rng(7)
    u0 = 1.0
    init = rng.standard_normal((m * NT + 1, 1))
    # Parareal: U^{k+1}_c = G(U^{k+1}_{c-1}) + F(U^k_{c-1}) - G(U^k_{c-1}), F = phi^m, G = phic
    U = init[::m, 0].copy()
    U[0] = u0
    snaps = []
    mgrit.mgrit(levels, np.array([u0]), gamma=0, tol=0.0, max_iter=4, tol_relative=False,
                u_init=init, callback=lambda k, u: snaps.append(u[::m, 0].copy()))
    for k in range(1, 5):
        Unew = U.copy()
        for c in range(1, NT + 1):
            Unew[c] = phic * Unew[c - 1] + phi**m * U[c - 1] - phic * U[c - 1]
        U = Unew
        # after k corrections and the following F-relaxation
        assert np.abs(snaps[k] - U).max() <= 1e-13 * np.abs(U).max()


def test_one_level_and_m1(meshes, model):
    P1 = MachineProblem(meshes, model, 32, 5e-3, (0,), ())
    useq = P1.sequential()
    u, _ = P1.mgrit(gamma=1)
    assert np.abs(u - useq).max() <= 1e-15 * np.abs(useq).max()
    # two levels, m = 1: the coarse propagator is the fine one and the coarse solve is exact
    Pm = MachineProblem(meshes, model, 32, 5e-3, (0, 0), (1,))
    u, h = Pm.mgrit(gamma=0, tol=1e-13, max_iter=3)
    assert np.abs(u - useq).max() <= 1e-13 * np.abs(useq).max()
    assert h[1] <= 1e-13 * h[0]


@pytest.mark.parametrize("gamma", [0, 1])
def test_exactness(meshes, model, gamma):
    N, m = 64, 4
    NT = N // m
    P = MachineProblem(meshes, model, N, 5e-3, (0, 0), (m,))
    useq = P.sequential()
    scale = np.abs(useq).max()
    front = []

    def cb(k, u):
        err = np.abs(u[::m] - useq[::m]).max(axis=1)
        exact = np.nonzero(err > 1e-11 * scale)[0]
        front.append(NT if exact.size == 0 else exact[0] - 1)

    need = NT if gamma == 0 else NT // 2
    u, h = P.mgrit(gamma=gamma, tol=0.0, max_iter=need, tol_relative=False, callback=cb)
    assert np.abs(u - useq).max() <= 1e-11 * scale
    # exact front after k corrections and the following relaxation: each coarse
    # correction adds one exact C-point, each FCF relaxation one more
    for k, f in enumerate(front):
        assert f >= min(NT, k * (1 + gamma) + gamma), front


@pytest.mark.parametrize("mode", [0, 2])
def test_spatial_coarsening_fixed_point(meshes, model, mode):
    P = MachineProblem(meshes, model, 128, 5e-3, (1, 0), (16,), residual_mode=mode)
    useq = P.sequential()
    u, h = P.mgrit(gamma=1, tol=1e-13, max_iter=30)
    assert h[-1] <= 1e-13 * h[0]
    assert rel_err_per_point(u, useq).max() <= 1e-10


def test_three_level_vcycle(meshes, model):
    P = MachineProblem(meshes, model, 128, 5e-3, (1, 1, 0), (4, 4))
    useq = P.sequential()
    u, h = P.mgrit(gamma=1, tol=1e-12, max_iter=30)
    assert len(h) - 1 < 16  # far faster than the exactness bound N/(2m) = 16
    assert rel_err_per_point(u, useq).max() <= 1e-9
