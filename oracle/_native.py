"""Build and load the oracle's plain-C core (liboracle.c) with gcc, via ctypes.

Test infrastructure only (see oracle/__init__.py).  The shared object is built in
place next to the source, with strict IEEE double arithmetic (no contraction into
fused multiply-adds, no fast-math) and OpenMP over independent targets.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "liboracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_handle = None


def build(force: bool = False) -> str:
    """Compile liboracle.so if it is missing or older than its source."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_P = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_d = ctypes.c_double
_i = ctypes.c_int


def lib():
    global _handle
    with _lock:
        if _handle is None:
            h = ctypes.CDLL(build())
            h.orc_direct_sum.argtypes = [_i, _P, _P, _P, _I, _i, _P, _d, _d, _i, _I, _P]
            h.orc_field.argtypes = [_i, _P, _P, _P, _i, _P, _d, _d, _i, _P, _P]
            h.orc_modes_trapezoid.argtypes = [_d, _i, _P, _P, _P, _P, _P, _d, _d, _i, _d, _P, _I]
            h.orc_modes_graded.argtypes = [_d, _i, _P, _P, _P, _P, _P, _d, _d, _i, _d, _i, _P, _P, _P]
            h.orc_kernel_ring.argtypes = [_d, _d, _d, _d, _d, _d, _d, _d, _d, _P]
            h.orc_kernel_xyz.argtypes = [_P, _P, _P, _d, _d, _P]
            for f in (h.orc_direct_sum, h.orc_field, h.orc_modes_trapezoid, h.orc_modes_graded,
                      h.orc_kernel_ring, h.orc_kernel_xyz):
                f.restype = None
            _handle = h
    return _handle


def dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def iptr(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I)


def as_f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def as_c128_view(a) -> np.ndarray:
    """Complex array -> contiguous float64 view of interleaved (re, im)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64)
