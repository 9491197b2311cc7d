"""Multi-process host logic of bench.py on CPU (gloo, world size 2): each
rank times its own query batch; the job reports the sum of the ranks' units
over the slowest rank's time (weak scaling, no data-path collective)."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t, u = bench.aggregate(1.0 + rank, 100 * (rank + 1))
    out.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.0, 300), (1, 2.0, 300)]


def test_aggregate_single_process():
    import bench

    assert bench.aggregate(3.5, 42) == (3.5, 42)
