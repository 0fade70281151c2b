"""Scalar test problem u' = lambda u for the two-level error closed form.

Backward Euler with step dt gives phi = 1 / (1 - lambda dt); re-discretisation
on the coarse grid (Sec. 2.1) gives phi_c = 1 / (1 - lambda m dt).
"""

from __future__ import annotations

import numpy as np

from . import mgrit


class ScalarPhi:
    def __init__(self, lam: float, dt: float):
        self.phi = 1.0 / (1.0 - lam * dt)

    def __call__(self, u_prev, i):
        return self.phi * u_prev


def two_level(lam: float, dt: float, m: int, NT: int):
    fine = mgrit.Level(phi=ScalarPhi(lam, dt), N=m * NT, m=m, transfer=_Identity())
    coarse = mgrit.Level(phi=ScalarPhi(lam, m * dt), N=NT)
    return [fine, coarse]


class _Identity:
    def restrict_state(self, u):
        return u

    def restrict_residual(self, r):
        return r

    def prolong(self, e):
        return e


def cpoint_error_after_one_iteration(levels, e_in: np.ndarray, gamma: int) -> np.ndarray:
    """Run one two-level iteration (relax, residual, coarse correction) from a
    state whose C-point errors are e_in (e_in[0] = 0) and return the C-point
    errors afterwards.  The exact solution is u_i = phi^i u_0 with u_0 = 1."""
    fine = levels[0]
    m = fine.m
    N = fine.N
    exact = fine.phi.phi ** np.arange(N + 1)
    u = np.zeros((N + 1, 1))
    u[:, 0] = exact
    u[::m, 0] += e_in
    g = np.zeros_like(u)
    g[0] = u[0]
    mgrit.relax(fine, u, g, gamma)
    r = mgrit.cpoint_residual(fine, u, g)
    mgrit.coarse_correction(levels, 0, u, g, r, gamma)
    return u[::m, 0] - exact[::m]
