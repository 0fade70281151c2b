"""GB300-native MGRIT for a PWM-driven 2D eddy-current machine model.

The compute path lives in libmgrit_em.so (CUDA kernels for sm_103a behind the C
ABI of include/mgrit_em.h); `api` is a thin ctypes binding with the same names.
Importing this package loads nothing; `api.Context` loads the library and
raises if it has not been built.
"""

__all__ = ["api", "lib", "build"]
