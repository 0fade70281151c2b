"""The C ABI library builds, loads and exports every function include/mgrit_em.h declares
(CPU only: no compute call is made)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mgrit_em.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1912_03106_gb300 import build, lib

    if not os.path.exists(lib.LIB_PATH):
        build.build()
    return lib.LIB_PATH


def test_exports_every_declared_function(libpath):
    names = declared_functions()
    assert len(names) >= 20
    so = ctypes.CDLL(libpath)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_1912_03106_gb300 import lib

    assert set(declared_functions()) == set(lib.EXPORTED)
    lib.load()


def test_defaults_are_sane(libpath):
    from paper_1912_03106_gb300 import lib

    L = lib.load()
    so = lib.mg_solver_opts()
    L.mg_solver_defaults(ctypes.byref(so))
    assert so.cg_tol == 1e-13 and so.max_cg > 0 and so.precision == lib.MG_FP64
    # the last fields: a binding whose layout drifted from the header reads garbage here
    assert so.smoother == 0 and so.cheb_ratio == 30.0 and so.smooth == 5 and so.base_tiles == 0
    o = lib.mg_opts()
    L.mg_opts_defaults(ctypes.byref(o))
    assert o.levels == 2 and o.m[0] == 16 and o.relax == 1 and o.restrict_mode == 2
    assert o.solver.cheb_ratio == 30.0 and o.solver.newton_tol == 1e-8


def test_null_context_is_rejected(libpath):
    from paper_1912_03106_gb300 import lib

    L = lib.load()
    assert L.mg_finalize(None) == -1  # MG_EINVAL, no CUDA call made
    assert L.mg_num_dofs(None, 0) == -1


def test_choose_levels_heuristic():
    """Host-only decision of the temporal coarsening plan (no GPU call)."""
    from paper_1912_03106_gb300 import api

    ks = [16, 32, 64, 128, 256, 512, 1024]
    # throughput k / ms saturates at 256 columns
    ms = [1.0, 1.0, 1.0, 1.1, 1.9, 3.8, 7.6]
    levels, m = api.mg_choose_levels(ks, ms, 4096, max_levels=5)
    assert m[0] == 16 and levels == 5 and m[1:] == [2, 2, 2]
    # a wider saturation point gives a smaller first factor
    levels, m = api.mg_choose_levels(ks, [1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.9], 4096, max_levels=3)
    assert m == [8, 2] and levels == 3
    # the coarsest level keeps at least 2 intervals
    levels, m = api.mg_choose_levels([16], [1.0], 64, max_levels=8)
    assert m[0] == 4 and 64 // 4 // (2 ** (levels - 2)) >= 2
    with pytest.raises(api.L.MgError):
        api.mg_choose_levels([16], [1.0], 63)
