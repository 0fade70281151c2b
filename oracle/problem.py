"""Assemble the oracle's MGRIT levels for a synthetic machine workload.

Level l of an L-level hierarchy with factors m_0, m_1, ...: N_l = N / (m_0 ... m_{l-1})
intervals of size dt_l = T / N_l (re-discretisation with the coarse step, Sec. 2.1),
on mesh space_levels[l]; the forcing of level point i is that of fine point
i * m_0 ... m_{l-1}.
"""

from __future__ import annotations

import numpy as np

from . import fem, mgrit, pwm, stepper, transfer


class MachineProblem:
    def __init__(self, meshes, model, N: int, T: float, space_levels, m, nonlinear: bool = False,
                 residual_mode: int = 2, newton_tol: float = 1e-8):
        self.meshes = meshes
        self.model = model
        self.N = N
        self.T = T
        self.space_levels = tuple(space_levels)
        self.m = tuple(m)
        self.signs = pwm.sign_table(model.pwm, T, N)
        self.fe = {}
        for s in set(self.space_levels):
            self.fe[s] = fem.FEModel(meshes[s], model)
        self.levels = []
        stride = 1
        for l, s in enumerate(self.space_levels):
            Nl = N // stride
            dt = T / Nl
            forcing = stepper.Forcing(self.fe[s].F, model.pwm.J0, self.signs, stride)
            if nonlinear:
                phi = stepper.NewtonPhi(self.fe[s], dt, forcing, newton_tol)
            else:
                phi = stepper.LinearPhi(self.fe[s], dt, forcing)
            last = l == len(self.space_levels) - 1
            ml = None if last else self.m[l]
            tr = None
            if not last:
                sc = self.space_levels[l + 1]
                between = meshes[sc:s + 1]
                tr = transfer.SpaceTransfer(self.fe[s], self.fe[sc], between, residual_mode)
                if N // stride % ml:
                    raise ValueError("N must be divisible by the product of the coarsening factors")
            self.levels.append(mgrit.Level(phi=phi, N=Nl, m=ml, transfer=tr))
            if not last:
                stride *= ml

    @property
    def n(self) -> int:
        return self.fe[self.space_levels[0]].n

    def sequential(self, a0: np.ndarray | None = None) -> np.ndarray:
        a0 = np.zeros(self.n) if a0 is None else a0
        return stepper.sequential(self.levels[0].phi, self.N, a0)

    def mgrit(self, gamma: int, tol: float = 1e-10, max_iter: int = 100, a0=None, **kw):
        a0 = np.zeros(self.n) if a0 is None else a0
        return mgrit.mgrit(self.levels, a0, gamma=gamma, tol=tol, max_iter=max_iter, **kw)


def rel_err_per_point(u: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """e_i = ||u_i - ref_i|| / ||ref_i|| for i >= 1 (a_0 = 0 exactly)."""
    num = np.linalg.norm(u[1:] - ref[1:], axis=1)
    den = np.linalg.norm(ref[1:], axis=1)
    return num / np.where(den > 0, den, 1.0)
