"""Material, coil and PWM *parameters* of the synthetic machine (data only).

Materials (per region tag of `synth.annulus`):
  rotor conductor  sigma = 3.7e7 S/m, nu = nu0            (Brauer law when nonlinear)
  air gap          sigma = 0,         nu = nu0
  stator iron      sigma = 0,         nu = nu0 / 1000     (Brauer law when nonlinear)
  coil sectors     sigma = 0,         nu = nu0
with nu0 = 1 / (4 pi 1e-7).

Coils: sector s (centred at 60deg*s) carries phase (0, 2, 1, 0, 2, 1)[s] with
sign (+1, -1, +1, -1, +1, -1)[s], i.e. A+, C-, B+, A-, C+, B- around the bore.
The source current density in sector s is J_s(t) = sign_s * J0 * b_phase(t),
b_phase(t) in {-1, 0, +1} being the PWM switching function of that phase.

Nothing here evaluates the PWM signal or assembles anything.
"""

from __future__ import annotations

import dataclasses
import math

from .annulus import N_REGIONS, REGION_COIL0, REGION_GAP, REGION_IRON, REGION_ROTOR

NU0 = 1.0 / (4.0e-7 * math.pi)
SIGMA_ROTOR = 3.7e7

COIL_PHASE = (0, 2, 1, 0, 2, 1)
COIL_SIGN = (1, -1, 1, -1, 1, -1)

# Brauer-type reluctivity nu(b2) = k1 * exp(k2 * b2) + k3, b2 = |B|^2
BRAUER_K = (3.8, 2.17, 396.2)

LAW_LINEAR = 0
LAW_BRAUER = 1


@dataclasses.dataclass(frozen=True)
class Material:
    sigma: float
    nu: float
    law: int = LAW_LINEAR
    k1: float = 0.0
    k2: float = 0.0
    k3: float = 0.0


@dataclasses.dataclass(frozen=True)
class PwmSpec:
    """Three-phase PWM source parameters.

    J0        amplitude [A/m^2]
    f_ref     reference (fundamental) frequency [Hz]
    f_carrier carrier frequency [Hz]
    carrier   0 = sawtooth 2*frac(x) - 1, 1 = triangle 1 - 4*|frac(x) - 1/2|, x = f_carrier*t
    mod_index amplitude of the sine references
    """

    J0: float = 1.0e6
    f_ref: float = 50.0
    f_carrier: float = 5.0e3
    carrier: int = 1
    mod_index: float = 1.0


@dataclasses.dataclass
class MachineModel:
    materials: list  # Material per region tag
    coil_phase: list  # (region, phase, sign) triples
    pwm: PwmSpec


def machine_model(nonlinear: bool = False, pwm: PwmSpec | None = None) -> MachineModel:
    mats = [None] * N_REGIONS
    k1, k2, k3 = BRAUER_K
    if nonlinear:
        mats[REGION_ROTOR] = Material(SIGMA_ROTOR, NU0, LAW_BRAUER, k1, k2, k3)
        mats[REGION_IRON] = Material(0.0, NU0 / 1000.0, LAW_BRAUER, k1, k2, k3)
    else:
        mats[REGION_ROTOR] = Material(SIGMA_ROTOR, NU0)
        mats[REGION_IRON] = Material(0.0, NU0 / 1000.0)
    mats[REGION_GAP] = Material(0.0, NU0)
    for s in range(6):
        mats[REGION_COIL0 + s] = Material(0.0, NU0)
    coils = [(REGION_COIL0 + s, COIL_PHASE[s], COIL_SIGN[s]) for s in range(6)]
    return MachineModel(materials=mats, coil_phase=coils, pwm=pwm or PwmSpec())
