"""mg_add_transfer: the spatial transfer of MGRIT given as a CSR matrix (Sec. 3.4,
FE nodal interpolation between nested meshes; Sec. 2.2 spatial coarsening), on
the GPU against the oracle.

Two cases: the matrix of a red refinement, which must reproduce the transfer the
library composes from the refinement's parent map bit for bit, and a mesh that red
refinement does not produce (every triangle of the 1,104-DOF annulus split into
three at its centroid), solved by two-level MGRIT with spatial coarsening onto the
annulus and compared with the oracle given the same matrix.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from synth.model import PwmSpec, machine_model
from oracle import transfer
from oracle.problem import MachineProblem, rel_err_per_point

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1912_03106_gb300 import api  # noqa: E402

from test_oracle_transfer import node_matrix  # noqa: E402


def setup(meshes, model, refine=True, given=()):
    """A context with the meshes, their refinements (if refine) and the given
    transfers [(fine, coarse, node-space P)]."""
    ctx = api.Context(0)
    ids = [ctx.mg_add_mesh(m.xy, m.tri, m.region, m.dirichlet_nodes()) for m in meshes]
    if refine:
        for k in range(1, len(meshes)):
            ctx.mg_add_refinement(ids[k], ids[k - 1], meshes[k].parent)
    for fine, coarse, P in given:
        P = sp.csr_matrix(P)
        ctx.mg_add_transfer(ids[fine], ids[coarse], P.indptr, P.indices, P.data)
    for r, mat in enumerate(model.materials):
        ctx.mg_set_material(r, mat.sigma, mat.nu, mat.law, mat.k1, mat.k2, mat.k3)
    for region, phase, sign in model.coil_phase:
        ctx.mg_set_source(region, phase, sign)
    p = model.pwm
    ctx.mg_set_pwm(p.J0, p.f_ref, p.f_carrier, p.carrier, p.mod_index)
    return ctx, ids


def solve(ctx, ids, N, T, space, m, tol, max_iter=40):
    n = ctx.mg_num_dofs(ids[space[0]])
    out = torch.empty((N + 1, n), dtype=torch.float64, device="cuda")
    opts = api.mgrit_opts(levels=len(space), m=m, space_level=tuple(ids[s] for s in space), relax=1, tol=tol,
                          max_iter=max_iter)
    rc, st = ctx.mg_solve(N, T, torch.zeros(n, dtype=torch.float64, device="cuda"), out, opts, allow=(-7,))
    return rc, st, out


def test_matrix_of_the_refinement_gives_the_same_solve():
    ms = synth.mesh_hierarchy(2)
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    node_P = transfer.prolongation_nodes(ms[1].parent, ms[0].n_nodes)
    N, T = 128, 5e-3 / 2
    ctx_a, ids_a = setup(ms, model)
    ctx_b, ids_b = setup(ms, model, given=[(1, 0, node_P)])
    _, st_a, u_a = solve(ctx_a, ids_a, N, T, (1, 0), (16,), 1e-9)
    _, st_b, u_b = solve(ctx_b, ids_b, N, T, (1, 0), (16,), 1e-9)
    assert torch.equal(u_a, u_b) and st_a["res_hist"] == st_b["res_hist"]
    ctx_a.close()
    ctx_b.close()


def test_barycentric_split_follows_the_oracle():
    """Two-level FCF MGRIT, N = 64, m = 8, fine level on the split mesh (3,408 DOFs),
    coarse level on the annulus through the given P: residual history of the first
    iterations as the oracle's with the same matrix, result the sequential solution."""
    m0 = synth.mesh_hierarchy(1)[0]
    mb, par = synth.barycentric_split(m0)
    P = node_matrix(par, mb.n_nodes, m0.n_nodes)
    meshes = [m0, mb]
    model = machine_model(pwm=PwmSpec(J0=1e6, f_carrier=5e3))
    N, T = 64, 5e-3 / 4
    ctx, ids = setup(meshes, model, refine=False, given=[(1, 0, P)])
    rc, st, out = solve(ctx, ids, N, T, (1, 0), (8,), 1e-10)
    assert rc == 0, st["res_hist"]
    prob = MachineProblem(meshes, model, N, T, (1, 0), (8,), transfers={(1, 0): P})
    ref = prob.sequential()
    assert rel_err_per_point(out.cpu().numpy(), ref).max() <= 1e-10
    _, hist = prob.mgrit(gamma=1, tol=0.0, max_iter=3, tol_relative=False)
    h = np.array(st["res_hist"][:4])
    assert np.all(np.abs(h - np.array(hist[:4])) <= 1e-6 * np.array(hist[:4])), (h, hist)
    ctx.close()


def test_transfer_of_non_nested_nodes_is_refused():
    """A coarse node that is no fine node (here: every unit row removed) has no
    state to inject: MG_EINVAL before anything is built."""
    m0 = synth.mesh_hierarchy(1)[0]
    mb, par = synth.barycentric_split(m0)
    P = node_matrix(par, mb.n_nodes, m0.n_nodes).tolil()
    P[:m0.n_nodes] = 0.0
    P = P.tocsr()
    P.eliminate_zeros()
    ctx = api.Context(0)
    ids = [ctx.mg_add_mesh(m.xy, m.tri, m.region, m.dirichlet_nodes()) for m in (m0, mb)]
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_add_transfer(ids[1], ids[0], P.indptr, P.indices, P.data)
    assert e.value.status == -1
    good = node_matrix(par, mb.n_nodes, m0.n_nodes)
    cols = good.indices.copy()
    cols[7] = m0.n_nodes  # a column past the coarse nodes
    with pytest.raises(api.L.MgError) as e:
        ctx.mg_add_transfer(ids[1], ids[0], good.indptr, cols, good.data)
    assert e.value.status == -1
    ctx.close()
