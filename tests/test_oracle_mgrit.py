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


# ------------------------------------------------------------------ F-cycles and nested iterations

class _Pow:
    """u -> a^p u with a counter (exact coarse propagators: p = m^l)."""

    def __init__(self, a, calls):
        self.a = a
        self.calls = calls

    def __call__(self, u_prev, i):
        self.calls[0] += 1
        return self.a * u_prev


def _scalar_levels(lam, dt, m, N, L, exact_coarse=False, calls=None):
    calls = calls if calls is not None else [0]
    phi = 1.0 / (1.0 - lam * dt)
    levels = []
    for l in range(L):
        a = phi ** (m ** l) if exact_coarse else 1.0 / (1.0 - lam * dt * m ** l)
        last = l == L - 1
        levels.append(mgrit.Level(phi=_Pow(a, calls), N=N // m ** l, m=None if last else m,
                                  transfer=None if last else scalar._Identity()))
    return levels, calls


def test_fcycle_on_two_levels_is_the_vcycle():
    lv, _ = _scalar_levels(-50.0, 0.01, 4, 64, 2)
    u_v, h_v = mgrit.mgrit(lv, np.array([1.0]), gamma=1, tol=0.0, max_iter=3, tol_relative=False)
    u_f, h_f = mgrit.mgrit(lv, np.array([1.0]), gamma=1, tol=0.0, max_iter=3, tol_relative=False, cycle_kind="F")
    assert np.array_equal(u_v, u_f) and h_v == h_f


@pytest.mark.parametrize("gamma,bound", [(0, 64 // 4), (1, 64 // 8)])
def test_fcycle_exactness(gamma, bound):
    """F- and FCF-relaxation propagate exact values (Sec. 2.1): after N/m (F) or
    N/(2m) (FCF) iterations the F-cycle iterate is the sequential solution."""
    lv, _ = _scalar_levels(-50.0, 0.01, 4, 64, 3)
    u, _ = mgrit.mgrit(lv, np.array([1.0]), gamma=gamma, tol=0.0, max_iter=bound, tol_relative=False,
                       cycle_kind="F")
    exact = (1.0 / (1.0 + 50.0 * 0.01)) ** np.arange(65)
    assert np.abs(u[:, 0] - exact).max() <= 1e-13


def test_fcycle_work_per_iteration():
    """Three levels, FCF: an F-cycle iteration does exactly one extra level-1
    V-cycle body (relaxation, residual, FAS right-hand side on level 2, the
    sequential level-2 solve, post F-relaxation) beyond the V-cycle iteration."""
    m, N = 4, 64
    counts = {}
    for kind in ("V", "F"):
        lv, calls = _scalar_levels(-50.0, 0.01, m, N, 3)
        g = np.zeros((N + 1, 1))
        g[0] = 1.0
        u = np.zeros_like(g)
        u[0] = 1.0
        mgrit.relax(lv[0], u, g, 1)
        r = mgrit.cpoint_residual(lv[0], u, g)
        calls[0] = 0
        mgrit.coarse_correction(lv, 0, u, g, r, 1, kind)
        counts[kind] = calls[0]
    N1, N2 = N // m, N // m ** 2
    NT1 = N1 // m
    v_body = (2 * m - 1) * NT1 + NT1 + N2 + N2 + (m - 1) * NT1
    assert counts["F"] - counts["V"] == v_body


def test_nested_iterations_exact_with_exact_coarse_propagators():
    """With coarse propagators equal to phi^(m^l), every level's own problem has
    the fine solution at its points, so the nested-iteration guess is exact."""
    lam, dt, m, N = -30.0, 0.01, 4, 256
    lv, _ = _scalar_levels(lam, dt, m, N, 4, exact_coarse=True)
    u = mgrit.nested_guess(lv, np.array([1.0]), gamma=1)
    exact = (1.0 / (1.0 - lam * dt)) ** np.arange(N + 1)
    assert np.abs(u[:, 0] - exact).max() <= 1e-14
    _, hist = mgrit.mgrit(lv, np.array([1.0]), gamma=1, tol=0.0, max_iter=0, tol_relative=False, nested=True)
    assert hist[0] <= 1e-14


def test_nested_iterations_two_levels_closed_form():
    """Two levels: the guess at C-points is the coarse sequential solution
    phi_c^c u_0, and the F-points follow by fine steps from it."""
    lam, dt, m, N = -20.0, 0.01, 8, 64
    lv, _ = _scalar_levels(lam, dt, m, N, 2)
    u = mgrit.nested_guess(lv, np.array([2.0]), gamma=1)
    phi, phic = 1.0 / (1.0 - lam * dt), 1.0 / (1.0 - lam * dt * m)
    for i in range(N + 1):
        c, j = divmod(i, m)
        assert abs(u[i, 0] - 2.0 * phic ** c * phi ** j) <= 1e-14
