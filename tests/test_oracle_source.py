"""Pins of the oracle's source waveforms, Joule losses and loss-based stopping
(Sec. 3.3 start-up ramp, Sec. 4.1 reference source for nested iterations,
Eq. losses and the stopping rule of Sec. 5.1).  CPU only."""

import math

import numpy as np
import pytest

import synth
from synth.model import PwmSpec, machine_model
from oracle import fem, pwm, stepper
from oracle.problem import MachineProblem


@pytest.fixture(scope="module")
def mesh0():
    return synth.mesh_hierarchy(1)


def test_pwm_waveform_without_ramp_is_the_sign_table():
    spec = PwmSpec(J0=1e6, f_carrier=5e3)
    assert np.array_equal(pwm.waveform(spec, 5e-3, 256, 0, 0.0), pwm.sign_table(spec, 5e-3, 256).astype(float))


def test_ramp_closed_form():
    T, N, tr = 0.04, 400, 0.02
    a = pwm.ramp(T, N, tr)
    t = np.arange(N + 1) * T / N
    assert a[0] == 0.0
    assert abs(a[100] - 0.5) <= 1e-15  # t = tr / 2
    assert np.all(a[t >= tr] == 1.0)
    assert np.all(np.diff(a[t <= tr]) > 0)
    assert abs(a[50] - 0.5 * (1 - math.cos(math.pi * 0.25))) <= 1e-15


def test_reference_waveform_is_balanced_three_phase():
    spec = PwmSpec(J0=1e6, f_carrier=5e3)
    w = pwm.waveform(spec, 0.02, 1000, 1, 0.0)
    assert np.abs(w.sum(axis=1)).max() <= 1e-14
    assert abs(np.abs(w).max() - 1.0) <= 1e-3


def test_joule_losses_of_a_constant_rate(mesh0):
    """u_i = i dt v gives dA/dt = v at every step: P_i = v^T M_sigma v; a rate
    carried by non-conducting nodes only (away from the rotor) loses nothing."""
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    P = MachineProblem(mesh0, model, 16, 1e-3, (0,), ())
    fe = P.fe[0]
    rng = np.random.default_rng(0)
    v = rng.standard_normal(fe.n)
    u = np.outer(np.arange(17) * (1e-3 / 16), v)
    L = P.joule_losses(u)
    assert L[0] == 0.0
    want = v @ (fe.M @ v)
    assert np.abs(L[1:] - want).max() <= 1e-12 * want
    # nodes whose every incident element is non-conducting
    cond = np.asarray(abs(fe.M).sum(axis=1)).ravel() > 0
    w = np.where(cond, 0.0, v)
    u2 = np.outer(np.arange(17) * (1e-3 / 16), w)
    assert np.abs(P.joule_losses(u2)).max() == 0.0


def test_reference_nested_guess_starts_from_the_reference_coarse_solve(mesh0):
    """Two levels on one mesh: the C-points of the nested guess with the reference
    source are the coarse sequential solution driven by the sine reference."""
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    N, T, m = 64, 2e-3, 8
    P = MachineProblem(mesh0, model, N, T, (0, 0), (m,))
    P.mgrit(gamma=1, tol=0.0, max_iter=0, tol_relative=False, nested="reference")  # builds the reference levels
    fe = fem.FEModel(mesh0[0], model)
    wave = pwm.waveform(model.pwm, T, N, 1, 0.0)
    phi_c = stepper.LinearPhi(fe, T / (N // m), stepper.Forcing(fe.F, model.pwm.J0, wave, m))
    coarse = stepper.sequential(phi_c, N // m, np.zeros(fe.n))
    from oracle import mgrit as om

    guess = om.nested_guess(P._ref_levels, np.zeros(fe.n), 1)
    assert np.abs(guess[::m] - coarse).max() <= 1e-12 * np.abs(coarse).max()


def test_joule_stop_rule_semantics(mesh0):
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    P = MachineProblem(mesh0, model, 64, 2e-3, (0, 0), (8,))
    u, hist = P.mgrit(gamma=1, tol=1e-2, max_iter=20, stop="joule")
    assert hist[0] == float("inf")
    assert hist[-1] <= 1e-2
    assert all(h > 1e-2 for h in hist[:-1])


@pytest.mark.parametrize("m", [(8,), (4, 2)])
def test_joule_change_of_rescaled_rates(mesh0, m):
    """Sec. 5.1's stopping quantity on trajectories with known losses.  The old
    trajectory moves at a constant rate v, so P_i = P = v^T M_sigma v at every
    step; the new one moves at s_i v in step i, so P_i(new) = s_i^2 P.  At the
    finest C-points (multiples of m_0) the change is |s^2 - 1| / s^2, which tells
    apart the reading it states (relative to the new losses) from dividing by the
    old losses; the F-points carry a larger change (s = 3) that must not count."""
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    N, T = 32, 1e-3
    P = MachineProblem(mesh0, model, N, T, (0,) * (len(m) + 1), m)
    v = np.random.default_rng(5).standard_normal(P.n)
    dt = T / N
    m0 = m[0]
    s = np.full(N + 1, 3.0)
    c_scale = [1.1, 0.8, 1.3, 1.05, 0.95, 1.2, 0.9, 1.15]
    for c in range(1, N // m0 + 1):
        s[c * m0] = c_scale[c - 1]
    s[0] = 1.0
    u_old = np.outer(np.arange(N + 1) * dt, v)
    u_new = np.cumsum(np.outer(s * dt, v), axis=0)
    u_new -= u_new[0]  # u_0 = 0; step i moves by s_i dt v
    want = max(abs(s[c] ** 2 - 1) / s[c] ** 2 for c in range(m0, N + 1, m0))
    got = P.joule_change(u_old, u_new)
    assert abs(got - want) <= 1e-12 * want, (got, want)
    # the other readings give other values, so the pin separates them
    assert abs(max(abs(s[c] ** 2 - 1) for c in range(m0, N + 1, m0)) - want) > 0.05
    assert abs((3.0 ** 2 - 1) / 3.0 ** 2 - want) > 0.05
