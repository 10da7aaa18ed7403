"""The multi-GPU path of bench.py is replicas only: each rank steps its own
instance of the workload, seeded by `bench.replica_seed`, times it, and rank 0
reports the slowest rank's time and the sum of the particle-steps of all ranks
(`bench.reduce_replicas`).  Two gloo ranks on the CPU run that path end to end
with the FP64 oracle standing in for the CUDA library: each draws its own
particles of the 96 x 80 hybrid workload, steps them, counts the particles each
step pushes, and reduces.  The test then checks the reduction against the
per-rank values gathered separately, and that the replicas are independent
(different seeds, different particles) yet reproducible (a rank's seed redraws
its particles exactly)."""
import os
import sys
import time

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 3


def _checksum(ps):
    return float(sum(np.sum(p[k].astype(np.float64) * (1.0 + np.arange(len(p[k])) % 7))
                     for p in ps for k in ("cell", "xo", "yo", "ur")))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_2406_14512_gb300 import workloads
        cfg = workloads.config("small_hybrid")
        base = int(cfg["seed"])
        cfg["seed"] = bench.replica_seed(base, rank)
        cfg["capacity"] = int(cfg["n_pairs"] * 1.1) + 100_000     # as bench.py sizes it
        ps = workloads.particles(cfg, threads=1)
        again = workloads.particles(cfg, threads=1)
        reproducible = _checksum(ps) == _checksum(again)
        o = oracle.Oracle(cfg)
        for s in range(2):
            o.set_particles(s, ps[s])
        pushed = 0
        t0 = time.perf_counter()
        for _ in range(STEPS):
            pushed += o.count(0) + o.count(1)   # the particles this step pushes
            o.step(1)
        el = time.perf_counter() - t0
        (t_max,), (c_sum,) = bench.reduce_replicas([el], [float(pushed)], world)
        mine = (rank, cfg["seed"] - base, el, pushed, _checksum(ps), reproducible, t_max, c_sum)
        allv = [None] * world
        dist.all_gather_object(allv, mine)
        out.put(allv if rank == 0 else None)
    except Exception as e:  # report instead of leaving the parent waiting
        out.put(f"rank {rank}: {type(e).__name__}: {e}")
        raise
    finally:
        dist.destroy_process_group()


def test_replicas_step_and_reduce_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=300) for _ in ps]
    assert not any(isinstance(r, str) for r in res), res
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    allv = next(r for r in res if r is not None)
    rows = sorted(allv)
    assert [r[1] for r in rows] == [0, 1000]                 # one seed per rank
    assert all(r[3] > 0 and r[5] for r in rows)              # work done; draws reproducible
    assert rows[0][4] != rows[1][4]                          # independent particles
    t_max, c_sum = max(r[2] for r in rows), float(sum(r[3] for r in rows))
    for r in rows:                                           # every rank holds the reduction
        assert r[6] == pytest.approx(t_max, rel=0, abs=0)
        assert r[7] == c_sum
