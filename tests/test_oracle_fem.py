"""Pins of the oracle's P1 assembly and grid transfer (CPU only).

T5: symmetry, SPD, mass row sums, constants in the stiffness kernel.
T6: Galerkin identities P^T K_f P = K_c, P^T M_f P = M_c on nested meshes with
    inherited coefficients (an exact consequence of nested P1 spaces).
T7: radial Poisson problem on the annulus against its closed form, O(h^2).
"""

import math

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from synth.model import Material, MachineModel, PwmSpec, machine_model
from oracle import fem, transfer
from oracle.stepper import BandedSPD


@pytest.fixture(scope="module")
def meshes():
    return synth.mesh_hierarchy(3)


@pytest.fixture(scope="module")
def fes(meshes):
    model = machine_model()
    return [fem.FEModel(m, model) for m in meshes]


def test_mesh_counts(meshes):
    # 24 x 48 cells: 1,200 nodes, 2,304 triangles, 1,104 interior nodes; red refinement x4
    assert meshes[0].n_nodes == 1200 and meshes[0].n_tri == 2304
    assert meshes[1].n_tri == 4 * 2304 and meshes[2].n_tri == 16 * 2304
    assert [m.interior_nodes().size for m in meshes] == [1104, 4512, 18240]


def test_symmetric_spd_and_rowsums(fes):
    for fe in fes[:2]:
        for A in (fe.K, fe.M, fe.K_full, fe.M_full):
            d = abs(A - A.T).max()
            assert d <= 1e-15 * abs(A).max()
        # K 1 = 0 before Dirichlet elimination (gradients of a constant vanish)
        assert np.abs(fe.K_full @ np.ones(fe.n_nodes)).max() <= 1e-9 * abs(fe.K_full).max()
        # consistent mass: row sum of node i = sigma * (area of its patch) / 3
        patch = np.zeros(fe.n_nodes)
        for k in range(3):
            np.add.at(patch, fe.mesh.tri[:, k], fe.sigma_e * fe.area / 3.0)
        assert np.allclose(np.asarray(fe.M_full.sum(axis=1)).ravel(), patch, rtol=1e-13, atol=0)
        # L = M/dt + K is SPD: the banded Cholesky factorisation succeeds
        BandedSPD(fe.M / 1e-5 + fe.K)
        # ... and K alone too (Dirichlet on both circles)
        BandedSPD(fe.K)


def test_not_spd_is_rejected(fes):
    with pytest.raises(Exception):
        BandedSPD(-fes[0].K)


def test_total_area(fes, meshes):
    # the polygonal annulus area tends to pi (b^2 - a^2); red refinement keeps it exactly
    areas = [fe.area.sum() for fe in fes]
    assert abs(areas[0] - areas[1]) <= 1e-15 * areas[0] * 10
    assert abs(areas[0] - math.pi * (0.1**2 - 0.03**2)) < 0.01 * areas[0]


@pytest.mark.parametrize("fine,coarse", [(1, 0), (2, 1), (2, 0)])
def test_galerkin_identity(fes, meshes, fine, coarse):
    P = transfer.prolongation(fes[fine], fes[coarse], meshes[coarse:fine + 1])
    for Af, Ac in ((fes[fine].K, fes[coarse].K), (fes[fine].M, fes[coarse].M)):
        G = (P.T @ Af @ P).tocsr()
        assert abs(G - Ac).max() <= 1e-12 * abs(Ac).max()


def test_prolongation_reproduces_linear_functions(fes, meshes):
    # nodal interpolation is exact for functions linear on coarse elements: x, y
    P = (transfer.prolongation_nodes(meshes[2].parent, meshes[1].n_nodes)
         @ transfer.prolongation_nodes(meshes[1].parent, meshes[0].n_nodes))
    for k in range(2):
        assert np.abs(P @ meshes[0].xy[:, k] - meshes[2].xy[:, k]).max() <= 1e-16


def test_injection_index(fes, meshes):
    inj = transfer.injection_index(fes[2], fes[0], meshes[0:3])
    assert np.array_equal(meshes[2].xy[fes[2].dof[inj]], meshes[0].xy[fes[0].dof])


def _poisson_error(mesh, nu=2.0, c=5.0):
    model = MachineModel(materials=[Material(0.0, nu)] * synth.N_REGIONS, coil_phase=[], pwm=PwmSpec())
    fe = fem.FEModel(mesh, model)
    load = np.zeros(fe.n_nodes)
    for k in range(3):
        np.add.at(load, mesh.tri[:, k], c * fe.area / 3.0)
    a = BandedSPD(fe.K).solve(load[fe.dof])
    r = np.hypot(*mesh.xy[fe.dof].T)
    ra, rb = 0.03, 0.1
    c1 = c * (rb**2 - ra**2) / (4 * nu * math.log(rb / ra))
    c2 = c * ra**2 / (4 * nu) - c1 * math.log(ra)
    exact = -c * r**2 / (4 * nu) + c1 * np.log(r) + c2
    return np.abs(a - exact).max() / np.abs(exact).max()


def test_poisson_closed_form_second_order():
    # fresh structured meshes (boundary nodes on the circles, so the polygonal
    # domain error is O(h^2) as well); red refinement would keep the coarse polygon
    ms = [synth.annulus_mesh(12 * 2**k, 24 * 2**k, jitter=0.0) for k in range(4)]
    errs = [_poisson_error(m) for m in ms]
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    assert errs[-1] < 2e-3
    assert all(1.8 < q < 2.3 for q in rates), (errs, rates)


def test_phase_loads(fes):
    fe = fes[0]
    # sum_i F_s[i] = sum over the coils of phase s of sign * (coil area); a sector's own
    # load sums to its area
    for s in range(3):
        want = sum(sign * fe.area[fe.mesh.region == reg].sum()
                   for reg, ph, sign in fe.model.coil_phase if ph == s)
        assert abs(fe.F[:, s].sum() - want) <= 1e-15
    pos = fe.mesh.region == synth.REGION_COIL0  # sector 0, phase 0, sign +
    full = np.zeros(fe.n_nodes)
    full[fe.dof] = fe.F[:, 0]
    assert full.max() > 0
    sector_area = fe.area[pos].sum()
    assert abs(np.clip(full, 0, None).sum() - sector_area) <= 1e-12 * sector_area
