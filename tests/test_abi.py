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
    o = lib.mg_opts()
    L.mg_opts_defaults(ctypes.byref(o))
    assert o.levels == 2 and o.m[0] == 16 and o.relax == 1 and o.restrict_mode == 2


def test_null_context_is_rejected(libpath):
    from paper_1912_03106_gb300 import lib

    L = lib.load()
    assert L.mg_finalize(None) == -1  # MG_EINVAL, no CUDA call made
    assert L.mg_num_dofs(None, 0) == -1
