"""The multi-GPU path of bench.py is replicas only: each rank times its own
instance, rank 0 reports the slowest rank's time and the sum of the work.
This exercises that reduction with two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    el = [1.0 + rank, 0.5 + 0.25 * rank]
    cnt = [100.0 * (rank + 1), 10.0 * (rank + 1)]
    t, c = bench.reduce_replicas(el, cnt, world)
    out.put((rank, t, c))
    dist.destroy_process_group()


def test_replica_reduction_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, c in res:
        assert t == [2.0, 0.75]           # max over ranks
        assert c == [300.0, 30.0]         # sum over ranks
