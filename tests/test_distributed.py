"""The body-partitioned solve (paper_1406_0236_gb300.distributed) on two CPU ranks
with the gloo backend: the bodies are split in contiguous, work-balanced ranges, sigma
is all-gathered before each inter-body sum and the Gram-Schmidt dot products and norms
are all-reduced; with oracle-backed rank-local operators, the two-rank GMRES equals
the one-rank oracle solve."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_1406_0236_gb300.distributed import (Exchange, LocalOperator, gmres_distributed, partition_bodies,
                                               row_ranges, solve_partitioned)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    """Three bodies of different sizes (two shapes), two plane waves."""
    wl = W.uneven3(n_rhs=2)
    return wl


class OracleOperator(LocalOperator):
    """Rank-local pieces from the oracle: the inter-body sum of the owned targets against
    all sources, and the block-diagonal inverse applied to the owned rows."""

    def __init__(self, P, rows):
        self.P = P
        self.rows = rows

    def _full(self, local):
        f = np.zeros((self.P.N, local.shape[1]), dtype=np.complex128)
        f[self.rows[0]:self.rows[1]] = local
        return f

    def apply_local(self, sigma_full):
        r0, r1 = self.rows
        y = self.P.interbody(sigma_full, targets=np.arange(r0, r1, dtype=np.int32))
        return sigma_full[r0:r1] + self.P.local_inverse(self._full(y))[r0:r1]

    def rhs_local(self, v_local):
        r0, r1 = self.rows
        return -self.P.local_inverse(self._full(v_local))[r0:r1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import Problem, fields
    wl = _workload()
    P = Problem(wl)
    sizes = [b.shape.n_nodes for b in wl.bodies]
    parts = partition_bodies(sizes, world)
    rows = row_ranges(sizes, parts)
    ex = Exchange(dist, rows)
    op = OracleOperator(P, rows[rank])
    v = fields.plane_wave(P.nodes.x, wl.directions, wl.k)
    x_loc, it, conv, rel = solve_partitioned(op, ex, v[rows[rank][0]:rows[rank][1]], 1e-12, maxit=200)
    full = ex.allgather_rows(x_loc)
    out[rank] = (full, it, conv, parts)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_partitioned_solve_equals_one_rank_oracle_solve(world):
    """2 ranks: two body ranges; 3: one body each (uneven shares: the padded all-gather);
    4: more ranks than bodies, one rank owns nothing and still joins every collective."""
    from oracle import Problem, fields, gmres
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    x0, it0, c0, parts = out[0]
    for q in range(1, world):
        xq, itq, cq, _ = out[q]
        assert cq and itq == it0
        assert np.array_equal(xq, x0)                 # every rank holds the same gathered solution
    assert c0
    assert len(parts) == world and parts[0][0] == 0 and parts[-1][1] == 3
    assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
    if world == 4:
        assert parts[3] == (3, 3)
    wl = _workload()
    P = Problem(wl)
    v = fields.plane_wave(P.nodes.x, wl.directions, wl.k)
    for r in range(v.shape[1]):
        ref = gmres(P.apply, P.rhs(v[:, r]), 1e-13).x
        assert np.linalg.norm(x0[:, r] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_one_rank_partitioned_gmres_equals_oracle_gmres():
    """World size 1 through the same driver (a stand-in exchange that returns its input)."""
    from oracle import Problem, fields, gmres
    wl = _workload()
    P = Problem(wl)

    class Single(Exchange):
        def __init__(self):
            self.rows = [(0, P.N)]

        def allgather_rows(self, local):
            return local

        def allreduce_sum(self, a):
            return a

    v = fields.plane_wave(P.nodes.x, wl.directions, wl.k)
    x, it, conv, rel = gmres_distributed(OracleOperator(P, (0, P.N)), Single(), P.rhs(v), 1e-12, maxit=200)
    assert conv and np.all(rel <= 1e-12)
    for r in range(v.shape[1]):
        ref = gmres(P.apply, P.rhs(v[:, r]), 1e-13).x
        assert np.linalg.norm(x[:, r] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_partition_balances_pair_work():
    sizes = [4100, 9000, 1200, 7000, 7000, 300, 12000]
    N = sum(sizes)
    w = [n * (N - n) for n in sizes]
    for world in (1, 2, 3, 4, 7, 9):
        parts = partition_bodies(sizes, world)
        assert len(parts) == world
        assert parts[0][0] == 0 and max(e for _, e in parts) == len(sizes)
        assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
        loads = [sum(w[b:e]) for b, e in parts]
        # no contiguous split does better than the largest share, which is at least the mean
        assert max(loads) >= sum(w) / world - 1e-9
        assert max(loads) <= sum(w) / world + max(w)
    rr = row_ranges(sizes, partition_bodies(sizes, 3))
    assert rr[0][0] == 0 and rr[-1][1] == N


class _FailingOperator(OracleOperator):
    """Raises at its n-th apply: a rank that fails between two steps (nothing in flight)."""

    def __init__(self, P, rows, fail_at):
        super().__init__(P, rows)
        self.calls = 0
        self.fail_at = fail_at

    def apply_local(self, sigma_full):
        self.calls += 1
        if self.calls == self.fail_at:
            raise RuntimeError("injected rank failure")
        return super().apply_local(sigma_full)


def _failing_worker(rank, world, port, out):
    import datetime
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    from oracle import Problem, fields
    from paper_1406_0236_gb300.distributed import RankFailure
    wl = _workload()
    P = Problem(wl)
    sizes = [b.shape.n_nodes for b in wl.bodies]
    rows = row_ranges(sizes, partition_bodies(sizes, world))
    ex = Exchange(dist, rows)
    op = _FailingOperator(P, rows[rank], 3) if rank == 1 else OracleOperator(P, rows[rank])
    v = fields.plane_wave(P.nodes.x, wl.directions, wl.k)
    t0 = time.time()
    try:
        solve_partitioned(op, ex, v[rows[rank][0]:rows[rank][1]], 1e-12, maxit=200)
        out[rank] = ("finished", "", time.time() - t0)
    except RankFailure as e:
        out[rank] = ("rank_failure", str(e), time.time() - t0)
    except RuntimeError as e:
        out[rank] = ("error", str(e), time.time() - t0)
    # a failed rank leaves without tearing the group down; its sockets close with the process


def test_a_failed_rank_ends_the_others_collectives_with_an_error():
    """Failure detection on the host: rank 1 raises between two GMRES steps and exits;
    rank 0's next exchange ends with RankFailure (peer gone, or the group's 20 s timeout)
    instead of waiting forever."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    alive = [p.is_alive() for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert not any(alive), "a rank was still waiting after 120 s"
    assert out[1][0] == "error" and "injected" in out[1][1]
    assert out[0][0] == "rank_failure", out[0]
    assert "rank 0 of 2" in out[0][1]
    assert out[0][2] < 60.0
