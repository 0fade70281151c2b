"""Three-phase PWM switching functions, Sec. 3.2-3.3.

b_s(t) = sgn[r_s(t) - c(t)]                      (Eq. machine_pwm; sgn(0) = 0)
r_s(t) = mod_index * sin(2 pi f_ref t + phi_s)   (Eq. machine_reference_signal)
phi = (0, -2 pi / 3, -4 pi / 3)                   (the printed offsets, read as the
                                                   standard three-phase shifts)
c(t): sawtooth 2 (x - floor x) - 1               (Eq. machine_carrier_signal, x = f_c t)
      triangle 1 - 4 |(x - floor x) - 1/2|       (the sine-triangle comparison of Sec. 3.2)

The fine time grid is t_i = i T / N.  When the number of carrier periods in the
horizon, q = f_c T, is an integer, frac(x_i) = ((q i) mod N) / N is formed from
integers so that the carrier is exact.
"""

from __future__ import annotations

import math

import numpy as np


def carrier_phase(f_carrier: float, T: float, N: int) -> np.ndarray:
    q = f_carrier * T
    i = np.arange(N + 1, dtype=np.int64)
    if abs(q - round(q)) <= 1e-9 * max(1.0, abs(q)):
        return ((int(round(q)) * i) % N).astype(np.float64) / N
    x = f_carrier * (i * (T / N))
    return x - np.floor(x)


def carrier(f_carrier: float, T: float, N: int, kind: int) -> np.ndarray:
    ph = carrier_phase(f_carrier, T, N)
    if kind == 0:
        return 2.0 * ph - 1.0
    if kind == 1:
        return 1.0 - 4.0 * np.abs(ph - 0.5)
    raise ValueError("carrier kind must be 0 (sawtooth) or 1 (triangle)")


def reference(f_ref: float, mod_index: float, T: float, N: int) -> np.ndarray:
    """(N+1, 3) sine references at t_i."""
    t = np.arange(N + 1, dtype=np.float64) * (T / N)
    phi = np.array([0.0, -2.0 * math.pi / 3.0, -4.0 * math.pi / 3.0])
    return mod_index * np.sin(2.0 * math.pi * f_ref * t[:, None] + phi[None, :])


def sign_table(pwm, T: float, N: int) -> np.ndarray:
    """(N+1, 3) int8 table b_s(t_i) in {-1, 0, +1}."""
    r = reference(pwm.f_ref, pwm.mod_index, T, N)
    c = carrier(pwm.f_carrier, T, N, pwm.carrier)
    return np.sign(r - c[:, None]).astype(np.int8)


def ramp(T: float, N: int, t_ramp: float) -> np.ndarray:
    """Start-up factor alpha(t_i) of Sec. 3.3: 0.5 (1 - cos(pi t / t_ramp)) for
    t < t_ramp, 1 afterwards; t_ramp = 0 means no ramp.  (The printed argument
    pi t / 2 is read as pi t / t_ramp with t_ramp two electric periods, so that the
    factor rises from 0 to 1 over those periods.)"""
    t = np.arange(N + 1, dtype=np.float64) * (T / N)
    if t_ramp <= 0.0:
        return np.ones(N + 1)
    return np.where(t < t_ramp, 0.5 * (1.0 - np.cos(math.pi * t / t_ramp)), 1.0)


def waveform(pwm, T: float, N: int, kind: int = 0, t_ramp: float = 0.0) -> np.ndarray:
    """(N+1, 3) float64 source waveform per phase at t_i: alpha(t) b_s(t) for the
    PWM source (kind 0) or alpha(t) r_s(t) for the sine reference (kind 1), which
    Sec. 4.1 uses as the source while nested iterations build the initial guess."""
    base = sign_table(pwm, T, N).astype(np.float64) if kind == 0 else reference(pwm.f_ref, pwm.mod_index, T, N)
    return base * ramp(T, N, t_ramp)[:, None]
