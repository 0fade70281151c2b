"""ctypes declarations of the C ABI in include/mgrit_em.h (marshalling only).

Loading fails loudly if libmgrit_em.so has not been built: there is no
fallback implementation of any entry point.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# MGRIT_EM_LIB may name another build of the same library (e.g. a tuning variant)
LIB_PATH = os.environ.get("MGRIT_EM_LIB") or os.path.join(HERE, "libmgrit_em.so")

MG_OK = 0
STATUS = {
    0: "MG_OK",
    -1: "MG_EINVAL",
    -2: "MG_ENOMEM",
    -3: "MG_ECUDA",
    -4: "MG_ENOTSPD",
    -5: "MG_ECG_MAXIT",
    -6: "MG_ENEWTON",
    -7: "MG_EMGRIT_MAXIT",
    -8: "MG_ETIMEOUT",
    -9: "MG_ESTATE",
    -10: "MG_ESTALLED",
    -11: "MG_ENONFINITE",
}

MG_FP64 = 0
MG_FP32_REFINE = 1


class mg_solver_opts(C.Structure):
    _fields_ = [
        ("cg_tol", C.c_double),
        ("refine_tol", C.c_double),
        ("inner_tol", C.c_double),
        ("max_cg", C.c_int),
        ("max_refine", C.c_int),
        ("precision", C.c_int),
        ("cluster", C.c_int),
        ("tile", C.c_int),
        ("precond", C.c_int),
        ("smooth", C.c_int),
        ("omega", C.c_double),
        ("path", C.c_int),
        ("newton_tol", C.c_double),
        ("max_newton", C.c_int),
        ("max_halvings", C.c_int),
        ("newton_lin_tol", C.c_double),
        ("rows_per_block", C.c_int),
        ("coarse_rows_per_block", C.c_int),
        ("base_tiles", C.c_int),
        ("smoother", C.c_int),
        ("cheb_ratio", C.c_double),
        ("halo_fusion", C.c_int),
        ("base_cores", C.c_int),
    ]


class mg_stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("n_hist", C.c_int),
        ("res_hist", C.c_double * 64),
        ("t_setup", C.c_double),
        ("t_solve", C.c_double),
        ("step_solves", C.c_int64),
        ("batched_steps", C.c_int64),
        ("cg_iters", C.c_int64),
        ("worst_status", C.c_int32),
        ("launches", C.c_int64),
        ("newton_iters", C.c_int64),
    ]


class mg_opts(C.Structure):
    _fields_ = [
        ("levels", C.c_int),
        ("m", C.c_int * 8),
        ("space_level", C.c_int * 8),
        ("relax", C.c_int),
        ("tol", C.c_double),
        ("tol_relative", C.c_int),
        ("max_iter", C.c_int),
        ("restrict_mode", C.c_int),
        ("solver", mg_solver_opts),
        ("cycle", C.c_int),
        ("nested", C.c_int),
        ("stop_rule", C.c_int),
        ("step_tol_ratio", C.c_double),
    ]


_P = C.c_void_p
_I64 = C.c_int64
_D = C.c_double
_SIGNATURES = {
    "mg_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "mg_destroy": (None, [_P]),
    "mg_last_error": (C.c_char_p, [_P]),
    "mg_set_stream": (C.c_int, [_P, _P]),
    "mg_add_mesh": (C.c_int, [_P, C.POINTER(C.c_int), _I64, _P, _I64, _P, _P, _I64, _P]),
    "mg_add_refinement": (C.c_int, [_P, C.c_int, C.c_int, _P]),
    "mg_add_transfer": (C.c_int, [_P, C.c_int, C.c_int, C.c_int64, _P, _P, _P]),
    "mg_set_material": (C.c_int, [_P, C.c_int32, _D, _D, C.c_int, _D, _D, _D]),
    "mg_set_source": (C.c_int, [_P, C.c_int32, C.c_int, C.c_int]),
    "mg_set_pwm": (C.c_int, [_P, _D, _D, _D, C.c_int, _D]),
    "mg_set_ramp": (C.c_int, [_P, _D]),
    "mg_finalize": (C.c_int, [_P]),
    "mg_num_dofs": (_I64, [_P, C.c_int]),
    "mg_get_operators": (C.c_int, [_P, C.c_int, C.POINTER(_I64), _P, _P, _P, _P, _P]),
    "mg_pwm_table": (C.c_int, [_P, _I64, _D, _P]),
    "mg_solver_defaults": (None, [C.POINTER(mg_solver_opts)]),
    "mg_opts_defaults": (None, [C.POINTER(mg_opts)]),
    "mg_step": (C.c_int, [_P, C.c_int, _I64, _D, _I64, C.c_int, _I64, _I64, _P, _I64, _P, _I64, C.c_int,
                          C.POINTER(mg_solver_opts), C.POINTER(mg_stats)]),
    "mg_step_static": (C.c_int, [_P, C.c_int, _I64, _D, _I64, C.c_int, _I64, _I64, _P, _I64, _P, _I64, C.c_int,
                                 C.POINTER(mg_solver_opts), C.POINTER(mg_stats)]),
    "mg_sequential": (C.c_int, [_P, C.c_int, _I64, _D, _P, _P, C.POINTER(mg_solver_opts), C.POINTER(mg_stats)]),
    "mg_solve": (C.c_int, [_P, _I64, _D, _P, _P, C.POINTER(mg_opts), C.POINTER(mg_stats)]),
    "mg_solve_host": (C.c_int, [_P, _I64, _D, _P, _P, C.POINTER(mg_opts), C.POINTER(mg_stats)]),
    "mg_sequential_host": (C.c_int, [_P, C.c_int, _I64, _D, _P, _P, C.POINTER(mg_solver_opts),
                                     C.POINTER(mg_stats)]),
    "mg_smoother_weights": (C.c_int, [C.POINTER(mg_solver_opts), _D, C.c_int, C.POINTER(C.c_float)]),
    "mg_choose_levels": (C.c_int, [C.POINTER(_D), C.POINTER(_D), C.c_int, _I64, C.c_int, C.c_int, C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)]),
    "mg_plan_levels": (C.c_int, [_P, C.c_int, C.c_int, _I64, _D, C.c_int, C.POINTER(mg_opts), C.POINTER(_D)]),
    "mg_joule_losses": (C.c_int, [_P, C.c_int, _I64, _D, _P, _P]),
    "mg_autotune": (C.c_int, [_P, C.c_int, _I64, _D, C.c_int, C.POINTER(mg_solver_opts), C.POINTER(_D)]),
    "mg_batch_solve": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_I64), C.POINTER(_D), C.POINTER(_P),
                                 C.POINTER(_P), C.POINTER(mg_opts), C.c_int, _I64, C.POINTER(C.c_int),
                                 C.POINTER(mg_stats)]),
    "mg_solve_work_bytes": (C.c_int, [_P, _I64, C.POINTER(mg_opts), C.POINTER(_I64)]),
    "mg_release_work": (C.c_int, [_P]),
}

EXPORTED = tuple(_SIGNATURES)

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (once) and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
