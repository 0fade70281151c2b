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
                 residual_mode: int = 2, newton_tol: float = 1e-8, t_ramp: float = 0.0, transfers=None):
        """transfers: {(fine mesh index, coarse mesh index): node-space P_s} for pairs
        whose transfer is given as a matrix rather than by red refinements."""
        self.transfers = dict(transfers or {})
        self.meshes = meshes
        self.model = model
        self.N = N
        self.T = T
        self.space_levels = tuple(space_levels)
        self.m = tuple(m)
        self.nonlinear = nonlinear
        self.residual_mode = residual_mode
        self.newton_tol = newton_tol
        self.signs = pwm.waveform(model.pwm, T, N, 0, t_ramp)
        self.ref_wave = pwm.waveform(model.pwm, T, N, 1, t_ramp)
        self.fe = {}
        for s in set(self.space_levels):
            self.fe[s] = fem.FEModel(meshes[s], model)
        self.levels = self._levels(self.signs)
        self._ref_levels = None

    def _levels(self, wave):
        model, N, T, meshes = self.model, self.N, self.T, self.meshes
        nonlinear, residual_mode, newton_tol = self.nonlinear, self.residual_mode, self.newton_tol
        signs = wave
        levels = []
        stride = 1
        for l, s in enumerate(self.space_levels):
            Nl = N // stride
            dt = T / Nl
            forcing = stepper.Forcing(self.fe[s].F, model.pwm.J0, signs, stride)
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
                tr = transfer.SpaceTransfer(self.fe[s], self.fe[sc], between, residual_mode,
                                            node_P=self.transfers.get((s, sc)))
                if N // stride % ml:
                    raise ValueError("N must be divisible by the product of the coarsening factors")
            levels.append(mgrit.Level(phi=phi, N=Nl, m=ml, transfer=tr))
            if not last:
                stride *= ml
        return levels

    @property
    def n(self) -> int:
        return self.fe[self.space_levels[0]].n

    def sequential(self, a0: np.ndarray | None = None) -> np.ndarray:
        a0 = np.zeros(self.n) if a0 is None else a0
        return stepper.sequential(self.levels[0].phi, self.N, a0)

    def mgrit(self, gamma: int, tol: float = 1e-10, max_iter: int = 100, a0=None, nested=False, stop="residual",
              **kw):
        """nested: False, True (nested iterations with the PWM source) or
        "reference" (nested iterations with the sine reference as the source,
        Sec. 4.1); stop: "residual" or "joule" (maximal relative change of the
        Joule losses at C-points between two iterations, Sec. 5.1)."""
        a0 = np.zeros(self.n) if a0 is None else a0
        if nested == "reference":
            if self._ref_levels is None:
                self._ref_levels = self._levels(self.ref_wave)
            kw["u_init"] = mgrit.nested_guess(self._ref_levels, a0, gamma)
        elif nested:
            kw["nested"] = True
        if stop == "joule":
            kw["stop_fn"] = self.joule_change
        return mgrit.mgrit(self.levels, a0, gamma=gamma, tol=tol, max_iter=max_iter, **kw)

    def joule_losses(self, u: np.ndarray) -> np.ndarray:
        """P_loss(t_i) = d_i^T M_sigma d_i, d_i = (u_i - u_{i-1}) / dt (per unit depth,
        Eq. losses), for i = 1..N on the finest level; P(t_0) = 0."""
        fe = self.fe[self.space_levels[0]]
        dt = self.T / self.N
        d = np.diff(u, axis=0) / dt
        P = np.zeros(u.shape[0])
        P[1:] = np.einsum("ij,ij->i", d, (fe.M @ d.T).T)
        return P

    def joule_change(self, u_old: np.ndarray, u_new: np.ndarray) -> float:
        """max over C-points c >= 1 of |P_c(new) - P_c(old)| / |P_c(new)|."""
        m = self.m[0]
        pn = self.joule_losses(u_new)[m::m]
        po = self.joule_losses(u_old)[m::m]
        den = np.where(np.abs(pn) > 0, np.abs(pn), 1.0)
        return float(np.max(np.abs(pn - po) / den))


def rel_err_per_point(u: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """e_i = ||u_i - ref_i|| / ||ref_i|| for i >= 1 (a_0 = 0 exactly)."""
    num = np.linalg.norm(u[1:] - ref[1:], axis=1)
    den = np.linalg.norm(ref[1:], axis=1)
    return num / np.where(den > 0, den, 1.0)
