"""Pins of the oracle's spatial transfer given as a matrix (Sec. 3.4, FE nodal
interpolation between nested meshes; Sec. 2.2 spatial coarsening), on a mesh that
red refinement does not produce: each triangle of the 1,104-DOF annulus split into
three at its centroid.  CPU only."""

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from synth.model import PwmSpec, machine_model
from oracle import fem, transfer


def node_matrix(parents, n_fine, n_coarse):
    """P_s of nodal interpolation from per-node parent lists: weight 1 for a node
    on a coarse node, 1/3 on each vertex for a centroid (the P1 value there)."""
    rows, cols, vals = [], [], []
    for i, p in enumerate(parents):
        if p[0] == p[1] == p[2]:
            rows.append(i), cols.append(int(p[0])), vals.append(1.0)
        else:
            for q in p:
                rows.append(i), cols.append(int(q)), vals.append(1.0 / 3.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_fine, n_coarse))


@pytest.fixture(scope="module")
def bary():
    m0 = synth.mesh_hierarchy(1)[0]
    mb, par = synth.barycentric_split(m0)
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    fc, ff = fem.FEModel(m0, model), fem.FEModel(mb, model)
    P = node_matrix(par, mb.n_nodes, m0.n_nodes)
    return m0, mb, fc, ff, P


def test_split_mesh_is_nested_and_conforming(bary):
    m0, mb, fc, ff, P = bary
    assert mb.n_nodes == m0.n_nodes + m0.n_tri and mb.n_tri == 3 * m0.n_tri
    area_c, _ = fem.element_geometry(m0.xy, m0.tri)
    area_f, _ = fem.element_geometry(mb.xy, mb.tri)  # raises unless counter-clockwise
    assert abs(area_f.sum() - area_c.sum()) <= 1e-15 * area_c.sum()
    np.testing.assert_allclose(area_f.reshape(3, -1).sum(axis=0), area_c, rtol=1e-12)
    assert ff.n == fc.n + m0.n_tri  # the centroids are interior unknowns


def test_given_matrix_reproduces_linear_functions(bary):
    """Nodal P1 interpolation is exact on linear functions."""
    m0, mb, fc, ff, P = bary
    f = lambda xy: 3.0 * xy[:, 0] - 2.0 * xy[:, 1] + 0.5
    np.testing.assert_allclose(P @ f(m0.xy), f(mb.xy), rtol=0, atol=1e-15)


def test_given_matrix_gives_the_galerkin_operators(bary):
    """Nested P1 spaces with inherited coefficients: P^T K_f P = K_c, P^T M_f P = M_c."""
    m0, mb, fc, ff, P = bary
    T = transfer.SpaceTransfer(ff, fc, None, 2, node_P=P)
    for A_f, A_c in ((ff.K, fc.K), (ff.M, fc.M)):
        G = T.P.T @ A_f @ T.P
        assert abs(G - A_c).max() <= 1e-13 * abs(A_c).max()


def test_injection_is_read_from_the_unit_rows(bary):
    m0, mb, fc, ff, P = bary
    T = transfer.SpaceTransfer(ff, fc, None, 2, node_P=P)
    u = np.random.default_rng(0).standard_normal(ff.n)
    # state restriction = values at the coarse nodes, which keep their numbers
    full = np.zeros(mb.n_nodes)
    full[ff.dof] = u
    np.testing.assert_array_equal(T.restrict_state(u), full[fc.dof])


def test_matrix_of_a_red_refinement_equals_the_refinement_transfer():
    """The same transfer given as a matrix or by the refinement's parent map."""
    ms = synth.mesh_hierarchy(2)
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    fc, ff = fem.FEModel(ms[0], model), fem.FEModel(ms[1], model)
    node_P = transfer.prolongation_nodes(ms[1].parent, ms[0].n_nodes)
    A = transfer.SpaceTransfer(ff, fc, ms[0:2], 2)
    B = transfer.SpaceTransfer(ff, fc, None, 2, node_P=node_P)
    assert abs(A.P - B.P).max() == 0.0
    np.testing.assert_array_equal(A.inj, B.inj)
