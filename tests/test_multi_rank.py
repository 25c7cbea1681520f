"""Host logic of the multi-GPU bench on CPU: world_size 2 over gloo.

Samples shard with no data-path collective (replicas); the only collective is
the max over ranks of the timed region, as the bench computes it.
"""

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ids = bench.shard_samples(rank, world, 8)
    t = bench.max_over_ranks(float(rank + 1) * 1.5, world)
    bench.barrier(world)
    q.put((rank, ids.tolist(), t))
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ids0, t0), (r1, ids1, t1) = res
    assert set(ids0).isdisjoint(ids1) and len(ids0) == len(ids1) == 8
    assert t0 == t1 == 3.0
