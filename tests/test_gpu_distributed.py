"""The rank-local pieces of the body-partitioned solve on the GPU: hzb_interbody_bodies
(rows of B sigma for a body range) against the oracle's rows, and the partitioned
GMRES driver over the library's kernels (one rank, the exchange returning its input)
against the library's own FP64 solve."""
import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, rand_c, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 5e-6)])
def test_interbody_rows_of_a_body_range(precision, tol):
    require_gpu()
    from oracle import Problem
    wl = W.uneven3(n_rhs=3)
    s = gpu_solver(wl)
    P = Problem(wl)
    sig = rand_c((P.N, 3), 17)
    offs = np.concatenate([[0], np.cumsum([b.shape.n_nodes for b in wl.bodies])])
    for b0, b1 in ((0, 1), (1, 3), (2, 3), (0, 3)):
        got = s.interbody_bodies(sig, b0, b1, precision=precision)
        ref = P.interbody(sig, targets=np.arange(offs[b0], offs[b1], dtype=np.int32))
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() < tol * np.abs(ref).max(), (b0, b1)


def test_partitioned_driver_on_library_kernels():
    require_gpu()
    import torch
    from paper_1406_0236_gb300.distributed import Exchange, LibraryOperator, partition_bodies, row_ranges, \
        solve_partitioned
    wl = W.uneven3(n_rhs=2)
    s = gpu_solver(wl, tol=1e-12)
    sizes = [b.shape.n_nodes for b in wl.bodies]
    parts = partition_bodies(sizes, 1)
    rows = row_ranges(sizes, parts)

    class Single(Exchange):
        def __init__(self):
            self.rows = rows

        def allgather_rows(self, local):
            return local

        def allreduce_sum(self, a):
            return a

    x, _, _ = s.get_nodes()
    v = np.exp(1j * wl.k * (x @ wl.directions.T))
    vd = torch.from_numpy(v).cuda()
    op = LibraryOperator(s, parts[0], rows[0], precision=0)
    xd, it, conv, rel = solve_partitioned(op, Single(), vd, 1e-12, maxit=200)
    assert conv
    s.solve_data(v)
    assert rel_l2(xd.cpu().numpy(), s.get_density()) < 1e-10
