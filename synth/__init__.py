"""Seeded synthetic inputs for the PWM-driven annular machine model.

This package generates *data only*: node coordinates, triangles, region tags,
Dirichlet node lists, the node-parent map of red refinement, material and coil
tables, and workload descriptions.  It contains none of the method's arithmetic
(no assembly, no time stepping, no MGRIT, no grid-transfer weights, no PWM
evaluation).  Both the CPU oracle and the CUDA library consume what it makes.
"""

from .annulus import (  # noqa: F401
    Mesh,
    annulus_mesh,
    refine,
    barycentric_split,
    mesh_hierarchy,
    REGION_ROTOR,
    REGION_GAP,
    REGION_IRON,
    REGION_COIL0,
    N_REGIONS,
)
from .model import (  # noqa: F401
    Material,
    MachineModel,
    PwmSpec,
    machine_model,
    NU0,
)
from .workloads import Workload, WORKLOADS, workload  # noqa: F401
