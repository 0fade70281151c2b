"""Backward-Euler propagator Phi and sequential time stepping.

Sec. 2: the one-step method u_i = Phi_i(u_{i-1}) (Eq. mgrit_nonlinear_system)
and the sequential forward block solve of the block-bidiagonal system A u = g.
Sec. 3.1, Eq. discrete_system: backward Euler on M a' + K(a) a = f,
    (M / dt + K(a_i)) a_i = f_i + (M / dt) a_{i-1},
with the forcing evaluated at the new time t_i (the printed 1/Delta T on the
right-hand side is read as the level's own dt: a step of size dt has dt on
both sides).  f_i = J0 * sum_s b_s(t_i) F_s with the PWM switching functions.

Linear systems are solved with a banded Cholesky factorisation (SciPy / LAPACK
dpbtrf, dpbtrs), which also fails loudly if the matrix is not SPD.
Nonlinear steps (Sec. 5) use damped Newton started at a_{i-1}: the step
length starts at 1 and is halved while the residual norm would grow (at most
40 halvings; a residual that still grows then is a Newton failure).  The
iteration stops, taking the full correction, as soon as that correction
satisfies ||delta|| <= newton_tol * ||a + delta||.
Deeply saturated steps after a PWM switching event need 20-30 halvings in
their first iterations.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def to_banded_upper(A: sp.spmatrix):
    """Upper banded storage ab[u + i - j, j] = A[i, j] (j >= i) for dpbtrf."""
    A = sp.triu(A).tocoo()
    u = int(np.max(A.col - A.row)) if A.nnz else 0
    n = A.shape[0]
    ab = np.zeros((u + 1, n))
    ab[u + A.row - A.col, A.col] = A.data
    return ab


class BandedSPD:
    """Factor once, solve many: A = U^T U in banded form."""

    def __init__(self, A: sp.spmatrix):
        self.c = sla.cholesky_banded(to_banded_upper(A), lower=False)

    def solve(self, b: np.ndarray) -> np.ndarray:
        return sla.cho_solve_banded((self.c, False), b)


class Forcing:
    """f(t_i) = J0 * sum_s w_s(t_i) F_s on one mesh; `signs` is the (N+1, 3) source
    waveform of the finest time grid (the PWM table b_s, possibly times the start-up
    ramp, or the sine reference), fine index = level index * stride."""

    def __init__(self, F: np.ndarray, J0: float, signs: np.ndarray, stride: int = 1):
        self.F = F
        self.J0 = J0
        self.signs = signs
        self.stride = stride

    def __call__(self, i: int) -> np.ndarray:
        b = self.signs[i * self.stride].astype(np.float64)
        return self.J0 * (self.F @ b)


class LinearPhi:
    """Phi_i(u) = (M/dt + K)^{-1} (M/dt u + f(t_i)) on one space level."""

    def __init__(self, fe, dt: float, forcing):
        self.fe = fe
        self.dt = dt
        self.forcing = forcing
        self.Mdt = (fe.M / dt).tocsr()
        self.L = (self.Mdt + fe.K).tocsr()
        self.chol = BandedSPD(self.L)

    def __call__(self, u_prev: np.ndarray, i: int) -> np.ndarray:
        return self.chol.solve(self.Mdt @ u_prev + self.forcing(i))


class NewtonPhi:
    """Phi_i(u) solving F(a) = (M/dt)(a - u) + K(a) a - f(t_i) = 0 by Newton."""

    def __init__(self, fe, dt: float, forcing, newton_tol: float = 1e-8, max_newton: int = 100,
                 max_halvings: int = 40):
        self.fe = fe
        self.dt = dt
        self.forcing = forcing
        self.Mdt = (fe.M / dt).tocsr()
        self.tol = newton_tol
        self.max_newton = max_newton
        self.max_halvings = max_halvings
        self.last_iters = 0
        self.history = []  # residual norms of the last solve, one per Newton iterate

    def residual(self, a, u_prev, f):
        return self.Mdt @ (a - u_prev) + self.fe.stiffness_at(a) @ a - f

    def __call__(self, u_prev: np.ndarray, i: int) -> np.ndarray:
        f = self.forcing(i)
        a = u_prev.copy()
        R = self.residual(a, u_prev, f)
        self.history = [np.linalg.norm(R)]
        for it in range(1, self.max_newton + 1):
            J = (self.Mdt + self.fe.jacobian_at(a)).tocsr()
            delta = -BandedSPD(J).solve(R)
            a_new = a + delta
            R_new = self.residual(a_new, u_prev, f)
            if np.linalg.norm(delta) <= self.tol * np.linalg.norm(a_new):
                # converged: the full correction is taken even if rounding lets the
                # residual, already at its floor, grow slightly
                self.history.append(np.linalg.norm(R_new))
                self.last_iters = it
                return a_new
            step = 1.0
            halvings = 0
            # halve while the residual grows (or overflows to inf / nan)
            while not (np.linalg.norm(R_new) <= np.linalg.norm(R)) and halvings < self.max_halvings:
                step *= 0.5
                halvings += 1
                a_new = a + step * delta
                R_new = self.residual(a_new, u_prev, f)
            if not (np.linalg.norm(R_new) <= np.linalg.norm(R)):
                raise RuntimeError("Newton step does not reduce the residual after the maximal number of halvings")
            a, R = a_new, R_new
            self.history.append(np.linalg.norm(R))
        raise RuntimeError("Newton did not converge")


def sequential(phi, N: int, u0: np.ndarray, g: np.ndarray | None = None) -> np.ndarray:
    """Forward block solve of A u = g: u_0 = u0 (+ g_0), u_i = Phi_i(u_{i-1}) + g_i."""
    u = np.zeros((N + 1, u0.size))
    u[0] = u0 if g is None else g[0]
    for i in range(1, N + 1):
        u[i] = phi(u[i - 1], i)
        if g is not None:
            u[i] += g[i]
    return u
