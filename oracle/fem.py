"""P1 finite elements for sigma dA/dt - div(nu grad A) = J_s on the 2D section.

Follows Sec. 3.1 (Eq. system_eddy_current reduced to the A_z unknown with
prescribed coil currents, depth l_z = 1) and its spatial discretisation,
Eq. semi_discrete_system:  M a'(t) + K(a) a = f(t).

Per triangle T with area |T| and constant barycentric gradients
G = [grad lambda_1; grad lambda_2; grad lambda_3] (3 x 2):
  K_T = nu_T |T| G G^T                     (stiffness, reluctivity nu_T)
  M_T = sigma_T |T| / 12 * (1 + delta_ij)  (consistent mass, conductivity sigma_T)
  F_T = J_T |T| / 3 * (1, 1, 1)            (load of a constant current density)
Dirichlet condition A_z = 0 on both circles: the boundary rows and columns are
dropped, unknowns are the interior nodes in node order.

Nonlinear law (Brauer type): nu(b2) = k1 exp(k2 b2) + k3 with b2 = |grad a|^2 on
each element (|B| = |grad A_z| in 2D).  The residual of one element is
nu(b2) |T| G G^T a_T; its Jacobian is |T| [nu G G^T + 2 nu'(b2) (G g)(G g)^T]
with g = G^T a_T = grad a on T and nu' = d nu / d b2.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def element_geometry(xy: np.ndarray, tri: np.ndarray):
    """Areas |T| (n_tri,) and barycentric gradients G (n_tri, 3, 2)."""
    p = xy[tri]  # (T, 3, 2)
    d1 = p[:, 1] - p[:, 0]
    d2 = p[:, 2] - p[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    if not np.all(det > 0):
        raise ValueError("triangles must be counter-clockwise and non-degenerate")
    area = 0.5 * det
    G = np.empty((tri.shape[0], 3, 2))
    for k in range(3):
        a = p[:, (k + 1) % 3]
        b = p[:, (k + 2) % 3]
        # grad lambda_k is perpendicular to the opposite edge (a -> b), pointing at vertex k
        G[:, k, 0] = (a[:, 1] - b[:, 1]) / det
        G[:, k, 1] = (b[:, 0] - a[:, 0]) / det
    return area, G


def _scatter(tri: np.ndarray, Ae: np.ndarray, n: int) -> sp.csr_matrix:
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    return sp.csr_matrix((Ae.ravel(), (rows, cols)), shape=(n, n))


def stiffness_elements(area, G, nu_e):
    return nu_e[:, None, None] * area[:, None, None] * np.einsum("eik,ejk->eij", G, G)


def mass_elements(area, sigma_e):
    ref = (np.ones((3, 3)) + np.eye(3)) / 12.0
    return sigma_e[:, None, None] * area[:, None, None] * ref[None]


class FEModel:
    """Assembled P1 model of one mesh, restricted to the interior nodes.

    mesh       synth.annulus.Mesh
    model      synth.model.MachineModel (materials, coil table)
    Attributes (interior DOFs, n = number of interior nodes):
      K  (n x n) stiffness at the linear reluctivities
      M  (n x n) consistent mass
      F  (n x 3) phase load vectors: F[:, s] = sum over coils of phase s of sign * int phi_i
      dof        interior node ids
    """

    def __init__(self, mesh, model):
        self.mesh = mesh
        self.model = model
        self.n_nodes = mesh.n_nodes
        self.area, self.G = element_geometry(mesh.xy, mesh.tri)
        mats = model.materials
        self.sigma_e = np.array([mats[r].sigma for r in mesh.region], dtype=np.float64)
        self.nu_e = np.array([mats[r].nu for r in mesh.region], dtype=np.float64)
        self.law_e = np.array([mats[r].law for r in mesh.region], dtype=np.int32)
        self.k_e = np.array([[mats[r].k1, mats[r].k2, mats[r].k3] for r in mesh.region], dtype=np.float64)
        self.dof = mesh.interior_nodes()
        self.n = self.dof.size
        # node -> interior dof index (-1 on the Dirichlet boundary)
        self.node2dof = np.full(self.n_nodes, -1, dtype=np.int64)
        self.node2dof[self.dof] = np.arange(self.n)
        self.K_full = _scatter(mesh.tri, stiffness_elements(self.area, self.G, self.nu_e), self.n_nodes)
        self.M_full = _scatter(mesh.tri, mass_elements(self.area, self.sigma_e), self.n_nodes)
        self.K = self.restrict(self.K_full)
        self.M = self.restrict(self.M_full)
        F = np.zeros((self.n_nodes, 3))
        for region, phase, sign in model.coil_phase:
            sel = mesh.region == region
            for k in range(3):
                np.add.at(F[:, phase], mesh.tri[sel, k], sign * self.area[sel] / 3.0)
        self.F = F[self.dof]

    def restrict(self, A: sp.csr_matrix) -> sp.csr_matrix:
        return A[self.dof][:, self.dof].tocsr()

    # ---------------- nonlinear material law (Sec. 5) ----------------
    def full_vector(self, a: np.ndarray) -> np.ndarray:
        v = np.zeros(self.n_nodes)
        v[self.dof] = a
        return v

    def grad(self, a: np.ndarray) -> np.ndarray:
        """Element gradients g_T = G^T a_T, shape (n_tri, 2)."""
        aT = self.full_vector(a)[self.mesh.tri]  # (T, 3)
        return np.einsum("eik,ei->ek", self.G, aT)

    def nu_of(self, b2: np.ndarray):
        """nu(b2) and d nu / d b2 per element (linear elements: nu_e, 0)."""
        nu = self.nu_e.copy()
        dnu = np.zeros_like(nu)
        nl = self.law_e == 1
        k1, k2, k3 = self.k_e[nl, 0], self.k_e[nl, 1], self.k_e[nl, 2]
        with np.errstate(over="ignore", invalid="ignore"):
            e = np.exp(k2 * b2[nl])  # may overflow to inf for |B| > ~18 T
            t1 = np.where(k1 == 0.0, 0.0, k1 * e)  # k1 = 0: the law is nu = k3 exactly
            t2 = np.where(k1 == 0.0, 0.0, k1 * k2 * e)
        nu[nl] = t1 + k3
        dnu[nl] = t2
        return nu, dnu

    def stiffness_at(self, a: np.ndarray) -> sp.csr_matrix:
        """K(a): stiffness with the reluctivity evaluated at a."""
        g = self.grad(a)
        nu, _ = self.nu_of(np.sum(g * g, axis=1))
        return self.restrict(_scatter(self.mesh.tri, stiffness_elements(self.area, self.G, nu), self.n_nodes))

    def jacobian_at(self, a: np.ndarray) -> sp.csr_matrix:
        """d(K(a) a)/da = sum_T |T| [nu G G^T + 2 nu' (G g)(G g)^T]."""
        g = self.grad(a)
        nu, dnu = self.nu_of(np.sum(g * g, axis=1))
        Gg = np.einsum("eik,ek->ei", self.G, g)  # (T, 3)
        Je = stiffness_elements(self.area, self.G, nu)
        Je = Je + 2.0 * (dnu * self.area)[:, None, None] * np.einsum("ei,ej->eij", Gg, Gg)
        return self.restrict(_scatter(self.mesh.tri, Je, self.n_nodes))
