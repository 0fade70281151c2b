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
