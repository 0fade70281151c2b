"""FAS-MGRIT, Algorithm 1 (Sec. 2.1) with spatial coarsening (Sec. 2.2).

Notation: level l has N_l intervals, points i = 0..N_l, and the space-time
system A_l(u) = g with block rows u_0 = g_0, u_i - Phi_i(u_{i-1}) = g_i.
With coarsening factor m every m-th point is a C-point (T_c = c m dt).

  F-relaxation: u_{cm+j} = Phi(u_{cm+j-1}) + g_{cm+j},  j = 1..m-1, every interval c
  C-relaxation: u_{cm}   = Phi(u_{cm-1})   + g_{cm},    c = 1..N_l/m
  relaxation:   F, then gamma times CF  (gamma = 0: "F", gamma = 1: "FCF")
  residual at C-points:  r_c = g_{cm} - u_{cm} + Phi(u_{cm-1}),  r_0 = g_0 - u_0
  restriction (injection R_I in time, then R_s in space):
      u2_c = R_s(u_{cm}),  g2_c = R_s(r_c)
  FAS coarse right-hand side:  G = A_2(u2) + g2,
      G_0 = u2_0 + g2_0,  G_c = u2_c - Phi^(2)(u2_{c-1}) + g2_c
  coarse solve A_2(v) = G: one recursive cycle, or on the coarsest level the
      sequential forward solve v_0 = G_0, v_c = Phi^(2)(v_{c-1}) + G_c.  A V-cycle
      recurses once; an F-cycle (Sec. 2.1, Fig. v_f_cycle) solves the coarse
      system by an F-cycle followed by a V-cycle on the coarse level (a single
      solve when the coarse level is the coarsest)
  error e = P_s(v - u2); correction with ideal interpolation: u_{cm} += e_c,
      followed by F-relaxation (on the finest level that F-relaxation is the first
      step of the next iteration's relaxation, which computes the same values).

The driver repeats: relax, residual norm ||r|| = sqrt(sum_{c>=1} ||r_c||^2) on the
finest level (the discrete space-time L2 norm at C-points), stop if small,
else coarse-grid correction.

Nested iterations (Sec. 2.1, initial guess): solve the coarsest level's own
problem A_L(u) = (R_s u0, 0, ..., 0) sequentially, then level by level towards
the finest interpolate it to the C-points (P_s in space, the coarse points are
the C-points in time), F-relax, and on every level below the finest apply one
V-cycle; the finest level's interpolated and F-relaxed values are the initial
guess of the iterations.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Level:
    """One MGRIT level: its propagator, interval count, coarsening factor and the
    spatial transfer to the next coarser level (None on the coarsest)."""

    phi: object  # callable (u_prev, i) -> u_i
    N: int
    m: int | None = None
    transfer: object | None = None


def f_relax(lv: Level, u: np.ndarray, g: np.ndarray) -> None:
    m = lv.m
    for c in range(lv.N // m):
        for j in range(1, m):
            i = c * m + j
            u[i] = lv.phi(u[i - 1], i) + g[i]


def c_relax(lv: Level, u: np.ndarray, g: np.ndarray) -> None:
    m = lv.m
    for c in range(1, lv.N // m + 1):
        i = c * m
        u[i] = lv.phi(u[i - 1], i) + g[i]


def cpoint_residual(lv: Level, u: np.ndarray, g: np.ndarray) -> np.ndarray:
    m = lv.m
    NT = lv.N // m
    r = np.zeros((NT + 1,) + u.shape[1:])
    r[0] = g[0] - u[0]
    for c in range(1, NT + 1):
        i = c * m
        r[c] = g[i] - u[i] + lv.phi(u[i - 1], i)
    return r


def relax(lv: Level, u: np.ndarray, g: np.ndarray, gamma: int) -> None:
    f_relax(lv, u, g)
    for _ in range(gamma):
        c_relax(lv, u, g)
        f_relax(lv, u, g)


def sequential_solve(lv: Level, u: np.ndarray, g: np.ndarray) -> None:
    u[0] = g[0]
    for i in range(1, lv.N + 1):
        u[i] = lv.phi(u[i - 1], i) + g[i]


def coarse_correction(levels, l: int, u: np.ndarray, g: np.ndarray, r: np.ndarray, gamma: int,
                      kind: str = "V") -> None:
    lv, nx = levels[l], levels[l + 1]
    m = lv.m
    tr = lv.transfer
    u2 = tr.restrict_state(u[::m])
    g2 = tr.restrict_residual(r)
    G = np.empty_like(u2)
    G[0] = u2[0] + g2[0]
    for c in range(1, nx.N + 1):
        G[c] = u2[c] - nx.phi(u2[c - 1], c) + g2[c]
    v = u2.copy()
    if kind == "F" and l + 1 < len(levels) - 1:
        cycle(levels, l + 1, v, G, gamma, "F")
        cycle(levels, l + 1, v, G, gamma, "V")
    else:
        cycle(levels, l + 1, v, G, gamma, "V")
    u[::m] += tr.prolong(v - u2)


def cycle(levels, l: int, u: np.ndarray, g: np.ndarray, gamma: int, kind: str = "V") -> None:
    """One V- or F-cycle on level l (used as the coarse solve of level l-1)."""
    lv = levels[l]
    if l == len(levels) - 1:
        sequential_solve(lv, u, g)
        return
    relax(lv, u, g, gamma)
    r = cpoint_residual(lv, u, g)
    coarse_correction(levels, l, u, g, r, gamma, kind)
    f_relax(lv, u, g)


def nested_guess(levels, u0: np.ndarray, gamma: int = 1) -> np.ndarray:
    """Initial guess on levels[0] by nested iterations (see the module notes)."""
    L = len(levels)
    u0s = [np.asarray(u0, dtype=np.float64)]
    for l in range(L - 1):
        u0s.append(levels[l].transfer.restrict_state(u0s[-1][None])[0])
    gs = []
    for l, lv in enumerate(levels):
        gl = np.zeros((lv.N + 1,) + u0s[l].shape)
        gl[0] = u0s[l]
        gs.append(gl)
    v = np.zeros_like(gs[-1])
    sequential_solve(levels[-1], v, gs[-1])
    for l in range(L - 2, -1, -1):
        lv = levels[l]
        u = np.zeros_like(gs[l])
        u[::lv.m] = lv.transfer.prolong(v)
        u[0] = u0s[l]
        f_relax(lv, u, gs[l])
        if l > 0:
            cycle(levels, l, u, gs[l], gamma, "V")
        v = u
    return v


def residual_norm(r: np.ndarray) -> float:
    return float(np.sqrt(np.sum(r[1:] ** 2)))


def mgrit(levels, u0: np.ndarray, gamma: int = 1, tol: float = 1e-10, max_iter: int = 100,
          tol_relative: bool = True, u_init: np.ndarray | None = None, callback=None, cycle_kind: str = "V",
          nested: bool = False, stop_fn=None):
    """Solve A u = g with g = (u0, 0, ..., 0) on levels[0].

    Returns (u, history) where history[k] is the residual norm after the
    relaxation of iteration k (k coarse-grid corrections before it).
    `callback(k, u)` is called after each relaxation (before the norm test).
    cycle_kind "V" or "F"; nested: initial guess by nested iterations.
    stop_fn(u_old, u_new): when given, the stop test is stop_fn(previous
    relaxed iterate, this one) <= tol from the second iteration on (the history
    then holds these values, the first entry inf); the residual is not used.
    """
    if nested and len(levels) > 1:
        u_init = nested_guess(levels, u0, gamma)
    lv = levels[0]
    shape = (lv.N + 1,) + np.shape(u0)
    g = np.zeros(shape)
    g[0] = u0
    if u_init is None:
        u = np.zeros(shape)
    else:
        u = np.array(u_init, dtype=np.float64, copy=True)
    u[0] = u0
    if len(levels) == 1:
        sequential_solve(lv, u, g)
        return u, [0.0]
    hist = []
    prev = None
    for it in range(max_iter + 1):
        relax(lv, u, g, gamma)
        r = cpoint_residual(lv, u, g)
        if stop_fn is None:
            hist.append(residual_norm(r))
        else:
            hist.append(float("inf") if prev is None else stop_fn(prev, u))
            prev = u.copy()
        if callback is not None:
            callback(it, u)
        ref = hist[0] if (tol_relative and stop_fn is None) else 1.0
        if hist[-1] <= tol * ref or it == max_iter:
            break
        coarse_correction(levels, 0, u, g, r, gamma, cycle_kind)
    return u, hist
