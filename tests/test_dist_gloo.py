"""Multi-rank aggregation of bench.py on CPU with gloo (world size 2).

The batched-einsum path shards by replicas (no data-path collective); the
only cross-rank step is the timing aggregation: max step time over ranks and
the units of all ranks.  Each rank reports a different time; both must see
the max, and the value must count both ranks' units.
"""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms, value = bench.aggregate(dist, [10.0 + 5 * rank, 1.0 + rank], units_per_rank=2.0)
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == [15.0, 2.0]
        assert value == pytest.approx(2 * 2.0 / 15e-3)
