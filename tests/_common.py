"""Shared helpers of the GPU parity tests (oracle on one side, C ABI on the other)."""
import functools

import numpy as np
import pytest

import workloads as W


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def require_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


def gpu_solver(wl, precision=0, tol=1e-12, **kw):
    from paper_1406_0236_gb300 import Options, Solver
    opt = Options(precision=precision, gmres_tol=tol, **kw)
    s = Solver.from_workload(wl, opt)
    s.build_scattering_matrices()
    return s


@functools.lru_cache(maxsize=None)
def oracle_problem(name, **kw):
    from oracle import Problem
    return Problem(W.by_name(name, **kw))


def rel_l2(a, b) -> float:
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rand_c(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)
