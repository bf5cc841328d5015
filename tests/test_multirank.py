"""Multi-rank logic of bench.py on CPU with the gloo backend (world size 2): each
rank takes its own incident direction (independent problems, weak scaling), the
job time is the slowest rank's, and the whole-job rate counts every rank's solves."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    d = bench.rank_direction(rank)
    local_ms = 100.0 * (rank + 1)                    # rank 1 is the slow one
    mx = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (d.tolist(), mx, bench.whole_job_rate(3, 1, world, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_solve_independent_problems_and_report_the_slowest():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    d0, m0, v0 = out[0]
    d1, m1, v1 = out[1]
    assert m0 == m1 == 200.0
    assert abs(v0 - 2 * 3 / 0.2) < 1e-12 and v0 == v1
    assert np.allclose(d0, [[0, 0, 1]]) and not np.allclose(d0, d1)
    assert abs(np.linalg.norm(d1) - 1) < 1e-12
