"""GB300 (sm_103a) multibody axisymmetric Helmholtz BIE solver — Python binding.

A thin ctypes layer over the C ABI in include/hzb.h (libhzb.so, built in place by
`paper_1406_0236_gb300.build`).  Argument marshalling only: every step of the
setup, the operator apply, the solve and the field evaluation runs in the CUDA
kernels of the library.  There is no CPU fallback: importing this package loads
libhzb.so and raises if it is missing.

Method: Hao, Martinsson, Young, "An efficient and highly accurate solver for
multi-body acoustic scattering problems involving rotationally symmetric
scatterers" — combined-field BIE (Sec. 2), Fourier-mode Nystrom discretisation of
each body (Sec. 3.2), block-diagonal preconditioner with per-mode scattering
matrices and GMRES (Sec. 4).
"""
from .binding import (HZB_PREC_DOUBLE_FLOAT, HZB_PREC_FP64, HZB_PREC_MIXED_FP32, HZB_OPEN_SHELL, HZB_SPHERE, HZB_SPHEROID,
                      HzbError, Mlp, Options, Solver, Stats, lib, library_path)

__all__ = ["HZB_PREC_DOUBLE_FLOAT", "HZB_PREC_FP64", "HZB_PREC_MIXED_FP32", "HZB_SPHERE", "HZB_SPHEROID", "HZB_OPEN_SHELL",
           "HzbError", "Mlp", "Options", "Solver", "Stats", "lib", "library_path"]
