"""The C ABI library builds, loads and exports every function include/mgrit_em.h declares
(CPU only: no compute call is made)."""

import ctypes
import os
import re

import numpy as np
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
    assert so.halo_fusion == 0 and so.base_cores == 0
    o = lib.mg_opts()
    L.mg_opts_defaults(ctypes.byref(o))
    assert o.levels == 2 and o.m[0] == 16 and o.relax == 1 and o.restrict_mode == 2
    assert o.solver.cheb_ratio == 30.0 and o.solver.newton_tol == 1e-8


@pytest.mark.parametrize("ratio", [10.0, 30.0, 100.0])
@pytest.mark.parametrize("nu", [1, 2, 3, 5, 8])
def test_chebyshev_smoother_weights_are_minimax(libpath, nu, ratio):
    """The smoothing polynomial p(x) = prod_s (1 - w_s x) of the library's weights
    is the scaled Chebyshev polynomial of [a, b] = [lam/ratio, lam]: it
    equioscillates with modulus 1/T_nu((b+a)/(b-a)) at the nu+1 Chebyshev extrema
    of [a, b] (which only the right roots achieve), never exceeds that modulus on
    [a, b], and stays within (0, 1] on [0, a)."""
    from paper_1912_03106_gb300 import api

    lam = 2.46
    w = np.array(api.mg_smoother_weights(lam, nu, api.solver_opts(cheb_ratio=ratio)), dtype=np.float64)
    b, a = lam, lam / ratio
    z0 = (b + a) / (b - a)
    bound = 1.0 / np.cosh(nu * np.arccosh(z0))

    def p(x):
        return np.prod(1.0 - np.outer(x, w), axis=1)

    k = np.arange(nu + 1)
    xk = (b + a) / 2 + (b - a) / 2 * np.cos(k * np.pi / nu)
    pk = p(xk)
    assert np.allclose(np.abs(pk), bound, rtol=1e-4, atol=0), (pk, bound)
    assert np.all(np.sign(pk[:-1]) != np.sign(pk[1:]))  # alternating signs
    x = np.linspace(a, b, 20001)
    assert np.abs(p(x)).max() <= bound * (1 + 1e-4)
    x0 = np.linspace(0.0, a, 2001, endpoint=False)
    assert np.all(p(x0) > 0.0) and np.all(p(x0) <= 1.0 + 1e-6) and p(np.zeros(1))[0] == 1.0


def test_jacobi_smoother_weights_and_bad_input(libpath):
    from paper_1912_03106_gb300 import api, lib

    assert api.mg_smoother_weights(2.46, 4, api.solver_opts(smoother=1, omega=0.6)) == pytest.approx([0.6] * 4)
    # without a bound (lam = 0) Chebyshev falls back to omega
    assert api.mg_smoother_weights(0.0, 3, api.solver_opts(omega=0.7)) == pytest.approx([0.7] * 3)
    for lam, nu, kw in ((2.0, 0, {}), (2.0, 9, {}), (-1.0, 2, {}), (2.0, 2, dict(smoother=2)),
                        (2.0, 2, dict(cheb_ratio=1.0))):
        with pytest.raises(lib.MgError):
            api.mg_smoother_weights(lam, nu, api.solver_opts(**kw))


def test_header_is_plain_c(tmp_path):
    """include/mgrit_em.h is a C header: a C99 translation unit that includes it and
    calls into it compiles without warnings (no C++ types cross the boundary)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "mgrit_em.h"\n'
                   "int main(void) {\n"
                   "    mg_solver_opts so; mg_opts o; float w[5];\n"
                   "    mg_solver_defaults(&so); mg_opts_defaults(&o);\n"
                   "    return (int)mg_smoother_weights(&so, 2.0, 5, w) + o.levels;\n"
                   "}\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_struct_layout_matches_binding(tmp_path):
    """The ctypes structures of the binding have the header's size and field
    offsets (a C program built with the header prints them)."""
    import shutil
    import subprocess

    from paper_1912_03106_gb300 import lib

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"mg_solver_opts": lib.mg_solver_opts, "mg_opts": lib.mg_opts, "mg_stats": lib.mg_stats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mgrit_em.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('    printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f in cls._fields_:
            lines.append('    printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {(w[0], w[1]): int(w[2]) for w in (x.split() for x in out) if len(w) == 3}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])


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
    # any divisor, not only powers of two: 63 = 3 x 21 gives 21 intervals >= 16
    levels, m = api.mg_choose_levels([16], [1.0], 63, max_levels=2)
    assert levels == 2 and m == [3]
    with pytest.raises(api.L.MgError):  # a prime number of intervals has no qualifying factor
        api.mg_choose_levels([16], [1.0], 61)


def test_choose_levels_reproduces_the_printed_examples():
    """Every temporal coarsening choice the paper prints (tests/golden/
    temporal_coarsening_examples.txt, each with its source): with step times that
    grow linearly from `processors` columns on, the batch width at which throughput
    stops growing is the processor count, and the heuristic gives the paper's
    factors."""
    from paper_1912_03106_gb300 import api

    path = os.path.join(ROOT, "tests", "golden", "temporal_coarsening_examples.txt")
    rows = [ln.split(None, 5) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 2
    for n, p, lv, cm, want, _src in rows:
        p = int(p)
        ks = [p // 4, p // 2, p, 2 * p, 4 * p]
        ms = [1.0, 1.0, 1.0, 2.0, 4.0]  # flat below p, linear above: throughput peaks at p
        levels, m = api.mg_choose_levels(ks, ms, int(n), max_levels=int(lv), coarse_m=int(cm))
        assert levels == int(lv) and m == [int(x) for x in want.split(",")], (n, p, levels, m)


def test_choose_levels_reproduces_the_worked_example():
    """Sec. 4.1's example: a fine grid of 129 points, 16 processors and five levels
    give a first coarsening factor of 8 (16 intervals on the second level, eight
    points per processor) and factor 2 below, down to a coarsest grid of 3 points.
    Translated to one GPU, the processors are the batch width at which a batched
    step stops gaining throughput: step times growing linearly from 16 columns on
    make that width 16."""
    from paper_1912_03106_gb300 import api

    levels, m = api.mg_choose_levels([16, 32, 64], [1.0, 2.0, 4.0], 128, max_levels=5)
    assert levels == 5 and m == [8, 2, 2, 2]
    assert 128 // 8 // 2 // 2 // 2 + 1 == 3  # points on the coarsest grid
