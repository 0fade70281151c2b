"""Pins of the oracle's PWM source (Sec. 3.2-3.3), CPU only."""

import math

import numpy as np

from synth.model import PwmSpec
from oracle import pwm


def test_carrier_shapes_exact():
    # q = f_c T = 4 carrier periods over N = 16 steps: phase advances by 1/4 each step
    tri = pwm.carrier(200.0, 0.02, 16, 1)
    saw = pwm.carrier(200.0, 0.02, 16, 0)
    assert np.array_equal(tri[:5], [-1.0, 0.0, 1.0, 0.0, -1.0])
    assert np.array_equal(saw[:5], [-1.0, -0.5, 0.0, 0.5, -1.0])


def test_reference_three_phase():
    r = pwm.reference(50.0, 1.0, 0.02, 4)
    assert np.allclose(r[0], [0.0, -math.sqrt(3) / 2, math.sqrt(3) / 2], atol=1e-15)
    assert np.allclose(r[1], [1.0, -0.5, -0.5], atol=1e-15)  # t = T/4
    assert np.allclose(r.sum(axis=1), 0.0, atol=1e-14)  # balanced phases


def test_first_row_and_sgn_zero():
    b = pwm.sign_table(PwmSpec(f_carrier=5e3), 5e-3, 256)
    assert b.dtype == np.int8 and b.shape == (257, 3)
    assert np.array_equal(b[0], [1, 1, 1])  # r(0) = (0, -.866, .866) > c(0) = -1
    # zero reference: b = sgn(-c) and sgn(0) = 0 where the triangle crosses zero
    z = pwm.sign_table(PwmSpec(f_carrier=200.0, mod_index=0.0), 0.02, 16)
    assert np.array_equal(z[:5, 0], [1, 0, -1, 0, 1])


def test_average_tracks_reference():
    # over one carrier period, mean of sgn(r - c) = r for a uniform carrier and slowly
    # varying r (the defining property of PWM, Sec. 1 and Sec. 3.2)
    spp = 2000  # samples per carrier period
    fc, T = 5e3, 0.02
    N = int(fc * T) * spp
    for kind in (0, 1):
        b = pwm.sign_table(PwmSpec(f_carrier=fc, carrier=kind, mod_index=0.8), T, N).astype(float)
        r = pwm.reference(50.0, 0.8, T, N)
        nper = N // spp
        means = b[:-1].reshape(nper, spp, 3).mean(axis=1)
        mid = r[:-1].reshape(nper, spp, 3).mean(axis=1)
        # triangle: symmetric sampling, second-order error; sawtooth: trailing-edge
        # sampling lags by up to max|r'| * T_c / 2 = 0.8 * 2 pi 50 / 5e3 / 2 ~ 0.025
        assert np.abs(means - mid).max() < (0.005 if kind == 1 else 0.03)


def test_non_integer_phase_path():
    ph = pwm.carrier_phase(333.3, 0.01, 7)
    x = 333.3 * np.arange(8) * (0.01 / 7)
    assert np.allclose(ph, x - np.floor(x), atol=0)
