"""The seeded input recipe (CPU only): meshes, region tags, named workloads and the
batching workload's instances are reproducible and follow their stated recipe.
The GPU path and the oracle both consume these inputs, so a silent change here
would move both sides at once; these checks pin the inputs themselves."""

import math

import numpy as np

import synth
from synth import annulus
from synth.workloads import WORKLOADS, instances, workload


def test_meshes_are_reproducible():
    a, b = synth.mesh_hierarchy(2), synth.mesh_hierarchy(2)
    for ma, mb in zip(a, b):
        assert np.array_equal(ma.xy, mb.xy) and np.array_equal(ma.tri, mb.tri)
        assert np.array_equal(ma.region, mb.region)
    other = annulus.annulus_mesh(seed=1)
    assert not np.array_equal(other.xy, a[0].xy)  # the jitter is drawn from the seed


def test_jitter_stays_inside_the_annulus_and_boundary_is_exact():
    m = synth.mesh_hierarchy(1)[0]
    r = np.hypot(m.xy[:, 0], m.xy[:, 1])
    assert r.min() >= annulus.R_IN - 1e-15 and r.max() <= annulus.R_OUT + 1e-15
    d = m.dirichlet_nodes()
    assert np.allclose(np.minimum(abs(r[d] - annulus.R_IN), abs(r[d] - annulus.R_OUT)), 0.0, atol=1e-15)
    # counter-clockwise triangles with positive area
    p = m.xy[m.tri]
    area = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    assert area.min() > 0.0


def test_region_tags_follow_the_centroid_rule_on_the_coarsest_mesh():
    m = synth.mesh_hierarchy(1)[0]
    c = m.xy[m.tri].mean(axis=1)
    r = np.hypot(c[:, 0], c[:, 1])
    ang = np.degrees(np.arctan2(c[:, 1], c[:, 0])) % 360.0
    assert np.all(m.region[r < annulus.R_ROTOR] == annulus.REGION_ROTOR)
    assert np.all(m.region[(r >= annulus.R_ROTOR) & (r < annulus.R_GAP)] == annulus.REGION_GAP)
    coil = m.region >= annulus.REGION_COIL0
    assert np.all((r[coil] >= annulus.R_COIL_IN) & (r[coil] <= annulus.R_COIL_OUT))
    s = m.region[coil] - annulus.REGION_COIL0
    off = (ang[coil] - 60.0 * s + 180.0) % 360.0 - 180.0
    assert np.all(np.abs(off) <= annulus.COIL_HALF_WIDTH_DEG)
    assert sorted(set(s.tolist())) == list(range(6))  # all six sectors are present


def test_refined_children_inherit_the_parent_region():
    coarse, fine = synth.mesh_hierarchy(2)
    # every fine triangle lies inside one coarse triangle: its centroid's region
    # on the coarse mesh is the tag it carries
    counts = np.bincount(fine.region, minlength=annulus.N_REGIONS)
    assert np.array_equal(counts, 4 * np.bincount(coarse.region, minlength=annulus.N_REGIONS))
    # nested nodes: coarse node (i, j) is fine node (2i, 2j) at the same place
    nth_c, nth_f = coarse.nth, fine.nth
    for i, j in ((0, 0), (3, 7), (coarse.nr, nth_c - 1)):
        assert np.array_equal(coarse.xy[i * nth_c + j], fine.xy[2 * i * nth_f + 2 * j])


def test_named_workloads_are_consistent():
    for w in WORKLOADS.values():
        assert w.N % math.prod(w.m) == 0  # every MGRIT level has whole intervals
        assert len(w.m) == w.levels - 1
        # carrier periods per step: f_carrier * dt is a dyadic rational, so the PWM
        # phase of every step is exact in binary floating point
        x = w.f_carrier * w.T / w.N
        assert x * 2 ** 20 == int(x * 2 ** 20)
    w1 = workload("cfg1_linear_l2_N4096")
    assert (w1.fine_level, w1.space_levels, w1.N, w1.T, w1.m, w1.relax) == (2, (2, 0, 0), 4096, 20e-3, (16, 16), 1)


def test_instances_are_seeded_and_inside_the_recipe():
    a = instances(64, seed=0, mesh_levels=(0, 1, 2), Ns=(256, 512, 1024), T=5e-3, nonlinear_levels=(0,))
    b = instances(64, seed=0, mesh_levels=(0, 1, 2), Ns=(256, 512, 1024), T=5e-3, nonlinear_levels=(0,))
    c = instances(64, seed=1, mesh_levels=(0, 1, 2), Ns=(256, 512, 1024), T=5e-3, nonlinear_levels=(0,))
    assert a == b and a != c
    for inst in a:
        assert inst.mesh_level in (0, 1, 2) and inst.N in (256, 512, 1024) and inst.T == 5e-3
        assert inst.f_carrier in (5e3, 10e3, 20e3) and 0.5e6 <= inst.J0 <= 3e6
        assert not inst.nonlinear or inst.mesh_level == 0
    assert any(i.nonlinear for i in a) and any(not i.nonlinear for i in a)
