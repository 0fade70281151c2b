"""Accuracy model of the double-float operator products (CPU).

The FP64 form's Krylov update forms L z on the GPU from two FP32 arrays L = Lh + Ll
and FP32 arithmetic: exact rounded products with their FMA error terms, two-sum
accumulation of the rounded products, the rest summed in FP32, one FP64 addition at
the end.  This test runs the same sequence of IEEE single-precision operations in
numpy (float32 rounding; an FMA is an exact float64 product rounded once to float32,
which is what a single-precision FMA computes) on rows of the 18,240-DOF step
operator with a smooth z, and checks the error bound the library relies on when it
uses these products for tolerances >= 1e-8: within 2^-43 of sum_j |L_ij z_j| (the
emulation gives about 2^-45.7 at worst), while FP64 summation stays near 2^-51.
The GPU kernel itself is checked against the oracle in test_gpu_graph_variants.py.
"""

import numpy as np

import synth
from synth.model import PwmSpec, machine_model
from oracle import fem

f32 = np.float32


def fma32(a, b, c):
    return f32(float(a) * float(b) + float(c))


def df_dot(vals, zs):
    hi = f32(0.0)
    lo = f32(0.0)
    for a, z in zip(vals, zs):
        ah = f32(a)
        al = f32(a - float(ah))
        p = f32(ah * z)
        pe = f32(float(ah) * float(z) - float(p))  # exact: ah * z = p + pe
        s = f32(hi + p)
        bp = f32(s - hi)
        err = f32(f32(hi - f32(s - bp)) + f32(p - bp))  # two-sum
        hi = s
        lo = fma32(al, z, f32(lo + f32(err + pe)))
    return float(hi) + float(lo)


def test_double_float_products_stay_within_the_bound():
    meshes = synth.mesh_hierarchy(3)
    fe = fem.FEModel(meshes[2], machine_model(pwm=PwmSpec(J0=1e6, f_carrier=20e3)))
    L = (fe.M / (20e-3 / 4096) + fe.K).tocsr()
    n = L.shape[0]
    rng = np.random.default_rng(0)
    z = (np.cumsum(rng.standard_normal(n)) * 1e-3 + 1e-4 * rng.standard_normal(n)).astype(np.float32)
    worst_df = worst_64 = worst_32 = 0.0
    for i in range(0, n, 23):
        cols = L.indices[L.indptr[i]:L.indptr[i + 1]]
        vals = L.data[L.indptr[i]:L.indptr[i + 1]]
        ref = np.sum(vals.astype(np.longdouble) * z[cols].astype(np.longdouble))
        scale = float(np.sum(np.abs(vals) * np.abs(z[cols].astype(np.float64))))
        if scale == 0.0:
            continue
        d64 = 0.0
        d32 = f32(0.0)
        for a, c in zip(vals, cols):
            d64 += a * float(z[c])
            d32 = fma32(f32(a), z[c], d32)
        worst_df = max(worst_df, float(abs(np.longdouble(df_dot(vals, z[cols])) - ref)) / scale)
        worst_64 = max(worst_64, float(abs(np.longdouble(d64) - ref)) / scale)
        worst_32 = max(worst_32, float(abs(np.longdouble(float(d32)) - ref)) / scale)
    assert worst_df <= 2.0 ** -43, np.log2(worst_df)
    assert worst_64 <= 2.0 ** -49, np.log2(worst_64)
    # the two-part form is what buys the accuracy: plain FP32 products are far worse
    assert worst_32 >= worst_df * 2.0 ** 15, (np.log2(worst_32), np.log2(worst_df))
