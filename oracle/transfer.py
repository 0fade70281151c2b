"""Spatial grid transfer between nested P1 meshes, Sec. 3.4 and Sec. 2.2.

P_s (prolongation) is standard FE (nodal) interpolation: a fine node that
coincides with a coarse node takes its value, a fine node at the midpoint of a
coarse edge takes the mean of the edge's two end values.  Across several
refinements P_s is the product of the single-level operators.  All operators act
on interior DOFs; Dirichlet values are zero.

Restrictions R_s (Algorithm 1, restriction step):
  state u:   nodal interpolation onto the coarse mesh = injection at coarse nodes
  residual:  mode 0  injection (nodal interpolation, as for the state)
             mode 1  P_s^T
             mode 2  D^{-1} P_s^T with D = diag(P_s^T 1)  (row-scaled transpose)
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def prolongation_nodes(parent: np.ndarray, n_coarse_nodes: int) -> sp.csr_matrix:
    """Node-space P (n_fine_nodes x n_coarse_nodes) of one red refinement."""
    nf = parent.shape[0]
    rows = np.repeat(np.arange(nf), 2)
    cols = parent.ravel()
    vals = np.full(2 * nf, 0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, n_coarse_nodes))  # duplicates sum to 1


def prolongation(fe_fine, fe_coarse, meshes_between) -> sp.csr_matrix:
    """Interior-DOF P_s from the coarse mesh to the fine mesh.

    meshes_between: [coarse, ..., fine] meshes, each (after the first) carrying
    its `parent` map into the previous one.
    """
    P = sp.identity(meshes_between[0].n_nodes, format="csr")
    for k in range(1, len(meshes_between)):
        Pk = prolongation_nodes(meshes_between[k].parent, meshes_between[k - 1].n_nodes)
        P = (Pk @ P).tocsr()
    return P[fe_fine.dof][:, fe_coarse.dof].tocsr()


def injection_index(fe_fine, fe_coarse, meshes_between) -> np.ndarray:
    """For each coarse interior DOF, the fine interior DOF at the same node."""
    node = np.arange(meshes_between[0].n_nodes)
    for k in range(1, len(meshes_between)):
        par = meshes_between[k].parent
        same = par[:, 0] == par[:, 1]
        inv = np.full(meshes_between[k - 1].n_nodes, -1, dtype=np.int64)
        inv[par[same, 0]] = np.nonzero(same)[0]
        node = inv[node]
    fine_node = node[fe_coarse.dof]
    idx = fe_fine.node2dof[fine_node]
    assert np.all(idx >= 0)
    return idx


def injection_from_matrix(node_P: sp.csr_matrix, fe_fine, fe_coarse) -> np.ndarray:
    """For each coarse interior DOF, the fine interior DOF at the same node, read
    from a node-space P_s of nested node sets: the fine node whose row of P_s is
    the coarse node's unit vector (nodal interpolation keeps coinciding values)."""
    P = node_P.tocsr()
    at = np.full(P.shape[1], -1, dtype=np.int64)
    for i in range(P.shape[0]):
        lo, hi = P.indptr[i], P.indptr[i + 1]
        if hi - lo == 1 and P.data[lo] == 1.0:
            at[P.indices[lo]] = i
    fine_node = at[fe_coarse.dof]
    assert np.all(fine_node >= 0), "coarse node that is not a fine node"
    idx = fe_fine.node2dof[fine_node]
    assert np.all(idx >= 0)
    return idx


class SpaceTransfer:
    """R_s / P_s between two MGRIT levels' space meshes (identity if equal).

    node_P: P_s given as a node-space matrix (fine nodes x coarse nodes) instead of
    the product of the red refinements in meshes_between."""

    def __init__(self, fe_fine, fe_coarse, meshes_between, residual_mode: int = 2, node_P=None):
        self.identity = fe_fine is fe_coarse
        self.mode = residual_mode
        if self.identity:
            return
        if node_P is None:
            self.P = prolongation(fe_fine, fe_coarse, meshes_between)
            self.inj = injection_index(fe_fine, fe_coarse, meshes_between)
        else:
            self.P = sp.csr_matrix(node_P)[fe_fine.dof][:, fe_coarse.dof].tocsr()
            self.inj = injection_from_matrix(node_P, fe_fine, fe_coarse)
        self.PT = self.P.T.tocsr()
        self.D = np.asarray(self.PT @ np.ones(self.P.shape[0])).ravel()

    def restrict_state(self, u: np.ndarray) -> np.ndarray:
        return u if self.identity else u[..., self.inj]

    def restrict_residual(self, r: np.ndarray) -> np.ndarray:
        if self.identity:
            return r
        if self.mode == 0:
            return r[..., self.inj]
        R = (self.PT @ r.T).T
        if self.mode == 2:
            R = R / self.D
        return R

    def prolong(self, e: np.ndarray) -> np.ndarray:
        return e if self.identity else (self.P @ e.T).T
