"""Parity on the two largest workloads at full size, on sampled outputs the oracle
computes one by one: 27 bodies of uneven sizes (64 right-hand sides) and 48 bodies
with open shells (about 2.2 million unknowns, 16 right-hand sides)."""
import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, rand_c, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _rows_of_modal_blocks(s, wl, body, rows, modes):
    from oracle import rings
    from oracle.modal import modal_rows
    shape = wl.bodies[body].shape
    rg = rings(shape)
    ref = modal_rows(rg, rows, wl.k, wl.eta)
    for p in modes:
        A = s.get_modal_block(body, p, 0, rg.n)
        assert np.abs(A[rows] - ref[p]).max() < 1e-11 * np.abs(ref[p]).max(), (body, p)


def _sampled_interbody(s, wl, R, nrows, seed, tol32, double_float=True):
    """FP32 kernel with all R right-hand sides, double-float kernel on the first one."""
    from oracle import Problem
    P = Problem(wl)
    assert s.N == P.N
    sig = rand_c((P.N, R), seed)
    rows = np.sort(np.random.default_rng(seed + 1).choice(P.N, nrows, replace=False)).astype(np.int32)
    ref = P.interbody(sig, targets=rows)
    y32 = s.interbody(sig, precision=1)
    assert rel_l2(y32[rows], ref) < tol32
    if double_float:
        ydf = s.interbody(np.ascontiguousarray(sig[:, :1]), precision=2)
        assert np.abs(ydf[rows, 0] - ref[:, 0]).max() < 1e-12 * np.abs(ref[:, 0]).max()


def test_mixed27_setup_and_interbody_rows():
    require_gpu()
    wl = W.mixed27()
    s = gpu_solver(wl)
    sizes = [b.shape.n_nodes for b in wl.bodies]
    big = int(np.argmax(sizes))
    _rows_of_modal_blocks(s, wl, big, np.array([0, 7, 150]), [0, 1, 30])
    _sampled_interbody(s, wl, 64, 12, 301, 5e-5)


def test_mixed48_shells_setup_and_interbody_rows():
    require_gpu()
    wl = W.mixed48()
    s = gpu_solver(wl)
    shell = next(q for q, b in enumerate(wl.bodies) if b.shape.kind == W.OPEN_SHELL)
    _rows_of_modal_blocks(s, wl, shell, np.array([0, 200, 383]), [0, 5, 60])
    _sampled_interbody(s, wl, 16, 8, 401, 8e-5, double_float=False)
