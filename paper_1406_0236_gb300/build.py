"""Build libhzb.so in place from csrc/ with nvcc for sm_103a.

Each translation unit compiles in its own process (in parallel), then nvcc links
the shared library.  Objects go to paper_1406_0236_gb300/_build/ (git-ignored).
Rebuilds only what is older than its sources or the shared headers.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhzb.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE]

SOURCES = ["api.cpp", "geometry.cpp", "setup.cu", "nbody.cu", "modal.cu", "krylov.cu", "mlp.cu", "noalloc.cu",
           "nbody_df.cu", "nbody_tc.cu", "nbody_sym.cu", "nbody_tc5.cu", "persist.cu", "modal_tma.cu", "compress.cu", "nbody_dfl.cu", "peaks.cu", "pod.cu", "modal_dfl.cu"]
# double-float error-free transformations must not be contracted into fused multiply-adds
# the FP32 inter-body kernel flushes denormals (irrelevant to its values, cheaper intrinsics)
PER_FILE = {"nbody_df.cu": ["-fmad=false"], "nbody_dfl.cu": ["-fmad=false"], "nbody.cu": ["-ftz=true"], "nbody_tc.cu": ["-ftz=true"], "nbody_sym.cu": ["-ftz=true"], "nbody_tc5.cu": ["-ftz=true"]}
HEADERS = ["hzb_internal.h", "curve.h", "kernel_math.cuh", "dfloat.cuh", "lean_df.cuh"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str, extra) -> str:
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    deps = [os.path.join(SRC, src)] + [os.path.join(SRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "hzb.h")]
    if os.path.exists(obj) and os.path.getmtime(obj) >= _newest(deps):
        return obj
    extra = list(extra) + PER_FILE.get(src, [])
    cmd = [nvcc()] + ARCH + FLAGS + list(extra) + ["-c", os.path.join(SRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc()] + ARCH + FLAGS + list(extra) + ["-x", "cu", "-c", os.path.join(SRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(OUT, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, len(SOURCES))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest(objs):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
