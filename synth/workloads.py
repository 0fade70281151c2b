"""Named workloads of the synthetic machine (data only).

Mesh levels: l0 = 24 x 48 cells (1,200 nodes, 1,104 interior DOFs), each next
level one red refinement (4,512 / 18,240 / 73,344 interior DOFs).

  cfg0_linear_l0_N256      l0, T = 5 ms,  N = 256,   5 kHz carrier, 2-level m=16 F-relax
  cfg1_linear_l2_N4096     l2, T = 20 ms, N = 4096,  20 kHz carrier, 3-level m=16 FCF,
                           coarse time levels on the l0 mesh (direct spatial coarsening)
  cfg2_mixed_l3_N16384     l3, T = 20 ms, N = 16384, 20 kHz, 3-level m=16 FCF, delayed spatial
                           coarsening: level 1 on l3, the coarsest level on l2
  cfg3_nonlinear_l2_N8192  l2 + Brauer law, J0 = 3e6, N = 8192, T = 20 ms, 3-level m=16 FCF
"""

from __future__ import annotations

import dataclasses


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    fine_level: int  # mesh level of MGRIT level 0
    space_levels: tuple  # mesh level per MGRIT level
    N: int
    T: float
    m: tuple  # coarsening factor per MGRIT level transition
    relax: int  # 0 = F, 1 = FCF
    f_carrier: float
    J0: float = 1.0e6
    nonlinear: bool = False
    precision: int = 0  # 0 = fp64, 1 = fp32 inner solves + fp64 refinement

    @property
    def levels(self) -> int:
        return len(self.space_levels)


WORKLOADS = {
    "cfg0_linear_l0_N256": Workload("cfg0_linear_l0_N256", 0, (0, 0), 256, 5.0e-3, (16,), 0, 5.0e3),
    "cfg1_linear_l2_N4096": Workload("cfg1_linear_l2_N4096", 2, (2, 0, 0), 4096, 20.0e-3, (16, 16), 1, 20.0e3),
    "cfg2_mixed_l3_N16384": Workload("cfg2_mixed_l3_N16384", 3, (3, 3, 2), 16384, 20.0e-3, (16, 16), 1, 20.0e3,
                                     precision=1),
    "cfg3_nonlinear_l2_N8192": Workload("cfg3_nonlinear_l2_N8192", 2, (2, 0, 0), 8192, 20.0e-3, (16, 16), 1, 20.0e3,
                                        J0=3.0e6, nonlinear=True),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


@dataclasses.dataclass(frozen=True)
class Instance:
    """One machine instance of the batching workload (data only)."""
    mesh_level: int
    N: int
    T: float
    f_carrier: float
    J0: float
    nonlinear: bool


def instances(count: int = 64, seed: int = 0, mesh_levels=(0, 1, 2, 3), Ns=(1024, 4096, 16384),
              carriers=(5.0e3, 10.0e3, 20.0e3), J0_range=(0.5e6, 3.0e6), T: float = 20.0e-3,
              nonlinear_fraction: float = 0.5, nonlinear_levels=None) -> list:
    """Seeded draw of uneven machine instances (the batching workload: mesh level,
    N, carrier and J0 drawn uniformly, linear / nonlinear by nonlinear_fraction).
    nonlinear_levels restricts which mesh levels may carry the nonlinear law."""
    import numpy as np

    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        lvl = int(rng.choice(mesh_levels))
        nl = bool(rng.random() < nonlinear_fraction)
        if nonlinear_levels is not None and lvl not in nonlinear_levels:
            nl = False
        out.append(Instance(lvl, int(rng.choice(Ns)), T, float(rng.choice(carriers)),
                            float(rng.uniform(*J0_range)), nl))
    return out
