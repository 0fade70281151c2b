"""Structured annulus meshes with seeded jitter and red refinement.

The mesh is logically a (nr+1) x nth grid of nodes in polar coordinates
(radial index i = 0..nr, angular index j = 0..nth-1, periodic in j).  Node
numbering is angular-fastest: node(i, j) = i * nth + j.  Each logical quad
(i, j) -> (i+1, j+1) is split along its (i, j)-(i+1, j+1) diagonal into a
"lower" triangle (i,j),(i+1,j),(i+1,j+1) and an "upper" triangle
(i,j),(i+1,j+1),(i,j+1); element index = 2*(i*nth + j) + {0 lower, 1 upper}.
Both triangles are counter-clockwise for the annulus orientation used here.

Red refinement (each triangle split into four through its edge midpoints,
straight edges) of such a mesh is again a structured mesh of the same kind on
the (2nr+1) x 2nth logical grid, with the same diagonal direction; coarse node
(i, j) becomes fine node (2i, 2j) and the new nodes sit at straight-edge
midpoints.  The refinement therefore produces exactly nested P1 spaces.
Children inherit their parent's region tag, so coefficients are piecewise
constant on the coarsest mesh at every level.

Region tags (coarsest mesh, decided by element centroid):
  rotor conductor  r < 0.055
  air gap          0.055 <= r < 0.06
  stator iron      r >= 0.06, except
  coil sector s    0.065 <= r <= 0.08 and |angle - 60deg*s| <= 15deg  (s=0..5)
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

REGION_ROTOR = 0
REGION_GAP = 1
REGION_IRON = 2
REGION_COIL0 = 3  # coil sector s has tag REGION_COIL0 + s, s = 0..5
N_REGIONS = REGION_COIL0 + 6

R_IN = 0.03
R_OUT = 0.1
R_ROTOR = 0.055
R_GAP = 0.06
R_COIL_IN = 0.065
R_COIL_OUT = 0.08
COIL_HALF_WIDTH_DEG = 15.0


@dataclasses.dataclass
class Mesh:
    """A structured annulus mesh (data only).

    xy       (n_nodes, 2) float64 node coordinates [m]
    tri      (n_tri, 3)   int32 node indices, counter-clockwise
    region   (n_tri,)     int32 region tags
    nr, nth  logical grid: nr radial cells, nth angular cells
    parent   (n_nodes, 2) int32 coarse-mesh parent nodes of each node (both
             entries equal for a node that coincides with a coarse node), or
             None on the coarsest mesh
    """

    xy: np.ndarray
    tri: np.ndarray
    region: np.ndarray
    nr: int
    nth: int
    parent: np.ndarray | None = None

    @property
    def n_nodes(self) -> int:
        return self.xy.shape[0]

    @property
    def n_tri(self) -> int:
        return self.tri.shape[0]

    def dirichlet_nodes(self) -> np.ndarray:
        """Nodes on r = R_IN (i = 0) and r = R_OUT (i = nr), where A_z = 0."""
        inner = np.arange(self.nth, dtype=np.int32)
        outer = self.nr * self.nth + np.arange(self.nth, dtype=np.int32)
        return np.concatenate([inner, outer])

    def interior_nodes(self) -> np.ndarray:
        """All nodes but the Dirichlet ones, in increasing order."""
        keep = np.ones(self.n_nodes, dtype=bool)
        keep[self.dirichlet_nodes()] = False
        return np.nonzero(keep)[0].astype(np.int32)


def _triangles(nr: int, nth: int) -> np.ndarray:
    i, j = np.meshgrid(np.arange(nr), np.arange(nth), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    jp = (j + 1) % nth
    a = i * nth + j
    b = (i + 1) * nth + j
    c = (i + 1) * nth + jp
    d = i * nth + jp
    tri = np.empty((nr * nth * 2, 3), dtype=np.int32)
    tri[0::2] = np.stack([a, b, c], axis=1)
    tri[1::2] = np.stack([a, c, d], axis=1)
    return tri


def _classify(xy: np.ndarray, tri: np.ndarray) -> np.ndarray:
    cen = xy[tri].mean(axis=1)
    r = np.hypot(cen[:, 0], cen[:, 1])
    ang = np.degrees(np.arctan2(cen[:, 1], cen[:, 0])) % 360.0
    region = np.full(tri.shape[0], REGION_IRON, dtype=np.int32)
    region[r < R_GAP] = REGION_GAP
    region[r < R_ROTOR] = REGION_ROTOR
    in_ring = (r >= R_COIL_IN) & (r <= R_COIL_OUT)
    for s in range(6):
        d = np.abs(((ang - 60.0 * s) + 180.0) % 360.0 - 180.0)
        region[in_ring & (d <= COIL_HALF_WIDTH_DEG)] = REGION_COIL0 + s
    return region


def annulus_mesh(nr: int = 24, nth: int = 48, jitter: float = 0.1, seed: int = 0) -> Mesh:
    """Coarsest mesh: r in [R_IN, R_OUT], interior nodes jittered.

    Each interior node (0 < i < nr) moves by U[-jitter, jitter] * h_r radially
    and U[-jitter, jitter] * h_theta in angle (numpy PCG64 stream from `seed`,
    drawn as an (n_interior, 2) array in node order).
    """
    hr = (R_OUT - R_IN) / nr
    hth = 2.0 * math.pi / nth
    r = R_IN + hr * np.arange(nr + 1, dtype=np.float64)
    th = hth * np.arange(nth, dtype=np.float64)
    rr, tt = np.meshgrid(r, th, indexing="ij")
    rr = rr.copy()
    tt = tt.copy()
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, size=((nr - 1) * nth, 2))
    rr[1:nr, :] += (jitter * hr) * u[:, 0].reshape(nr - 1, nth)
    tt[1:nr, :] += (jitter * hth) * u[:, 1].reshape(nr - 1, nth)
    xy = np.stack([(rr * np.cos(tt)).ravel(), (rr * np.sin(tt)).ravel()], axis=1)
    tri = _triangles(nr, nth)
    return Mesh(xy=xy, tri=tri, region=_classify(xy, tri), nr=nr, nth=nth, parent=None)


def refine(m: Mesh) -> Mesh:
    """Red refinement with straight-edge midpoints; see the module docstring."""
    nr, nth = m.nr, m.nth
    NR, NTH = 2 * nr, 2 * nth
    I, J = np.meshgrid(np.arange(NR + 1), np.arange(NTH), indexing="ij")
    I = I.ravel()
    J = J.ravel()
    # parent nodes on the coarse logical grid
    i0 = I // 2
    j0 = J // 2
    i1 = np.where(I % 2 == 1, i0 + 1, i0)
    j1 = np.where(J % 2 == 1, (j0 + 1) % nth, j0)
    p0 = (i0 * nth + j0).astype(np.int32)
    p1 = (i1 * nth + j1).astype(np.int32)
    parent = np.stack([p0, p1], axis=1)
    xy = 0.5 * (m.xy[p0] + m.xy[p1])
    tri = _triangles(NR, NTH)
    # region of each fine triangle = region of the coarse triangle containing it
    e = np.arange(tri.shape[0])
    q = e // 2
    upper = e % 2
    Iq = q // NTH
    Jq = q % NTH
    a = Iq % 2
    b = Jq % 2
    # lower fine tri centroid (a+2/3, b+1/3)/2, upper (a+1/3, b+2/3)/2 in coarse-local units;
    # coarse lower triangle covers angular-offset <= radial-offset
    cx = np.where(upper == 0, a + 2.0 / 3.0, a + 1.0 / 3.0)
    cy = np.where(upper == 0, b + 1.0 / 3.0, b + 2.0 / 3.0)
    parent_upper = (cy > cx).astype(np.int64)
    parent_e = 2 * ((Iq // 2) * nth + (Jq // 2)) + parent_upper
    region = m.region[parent_e].astype(np.int32)
    return Mesh(xy=xy, tri=tri, region=region, nr=NR, nth=NTH, parent=parent)


def barycentric_split(m: Mesh) -> tuple[Mesh, np.ndarray]:
    """Each triangle split into three at its centroid: a mesh nested in m (every
    node of m is a node of it, every triangle of m the union of three of its
    triangles) that red refinement does not produce.

    Returns (mesh, parents).  The nodes of m keep their numbers; the centroid of
    triangle e is node m.n_nodes + e.  Triangle e's children (a, b, c), (b, d, c),
    (d, a, c) for e = (a, b, d) with centroid c are numbered e, n_tri + e,
    2 n_tri + e and inherit its region.  nr, nth still describe the logical grid
    of m, so the Dirichlet nodes are unchanged (no centroid lies on a circle);
    `parent` is None (not a red refinement).  parents (n_nodes, 3) int32 lists for
    each node the nodes of m it lies on: (p, p, p) for node p of m, the three
    vertices of e for the centroid of e.
    """
    n = m.n_nodes
    xy = np.vstack([m.xy, m.xy[m.tri].mean(axis=1)])
    c = (n + np.arange(m.n_tri)).astype(np.int32)
    a, b, d = m.tri[:, 0], m.tri[:, 1], m.tri[:, 2]
    tri = np.concatenate([np.stack([a, b, c], axis=1), np.stack([b, d, c], axis=1),
                          np.stack([d, a, c], axis=1)]).astype(np.int32)
    region = np.tile(m.region, 3).astype(np.int32)
    parents = np.vstack([np.repeat(np.arange(n, dtype=np.int32)[:, None], 3, axis=1), m.tri]).astype(np.int32)
    return Mesh(xy=xy, tri=tri, region=region, nr=m.nr, nth=m.nth, parent=None), parents


def mesh_hierarchy(levels: int = 4, nr: int = 24, nth: int = 48, jitter: float = 0.1,
                   seed: int = 0) -> list[Mesh]:
    """[l0, l1, ...]: l0 is the jittered coarse annulus, l(k+1) = refine(l(k))."""
    out = [annulus_mesh(nr, nth, jitter, seed)]
    for _ in range(levels - 1):
        out.append(refine(out[-1]))
    return out
