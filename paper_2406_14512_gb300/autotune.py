"""Autotuner of the launch shape: tile size of the particle sort (and of the
tiled push's shared-memory region) and the sort cadence.

Candidates are timed on throwaway instances of an n x n sample of the
workload (same particles per cell, placement and momenta), each for a few
whole steps through the C ABI, including the amortised sort.  The tile with
its halo must fit the shared memory of one block, so large tiles are only
tried with short cadences.  Returns the fastest configuration and the full
table.  GPU only: the timings are CUDA events around graph-replayed steps.

    python -m paper_2406_14512_gb300.autotune --workload c3 --grid 1024
"""
from __future__ import annotations

import argparse
import json
import itertools

DEFAULT_TILES = [(8, 32), (16, 16), (16, 24), (16, 32), (32, 32)]
DEFAULT_CADENCES = [2, 4, 8]


def time_candidate(cfg: dict, ps, steps: int, warmup: int) -> float:
    """Milliseconds per whole step of one configuration (CUDA events)."""
    import torch
    from . import hff
    sim = hff.Sim(cfg)
    try:
        for s in range(2):
            sim.load(s, ps[s])
        sim.step(warmup)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(sim.stream)
        sim.step(steps)
        b.record(sim.stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps
    finally:
        sim.close()


def tune(workload: str = "c3", grid: int = 1024, tiles=None, cadences=None, steps: int = 16,
         warmup: int = 4, pairs: int = 0) -> dict:
    from . import hff, workloads
    base = workloads.sample(workload, grid)
    if pairs:
        base["n_pairs"] = pairs
    base["capacity"] = int(base["n_pairs"] * 1.1) + 10_000
    ps = workloads.particles(base)
    table = []
    for (tr, tt), k in itertools.product(tiles or DEFAULT_TILES, cadences or DEFAULT_CADENCES):
        cfg = dict(base, tile_r=tr, tile_t=tt, sort_every=k)
        try:
            ms = time_candidate(cfg, ps, steps, warmup)
        except hff.HffError as e:  # tile + halo larger than the shared memory of a block
            table.append({"tile_r": tr, "tile_t": tt, "sort_every": k, "ms_per_step": None, "error": str(e)})
            continue
        table.append({"tile_r": tr, "tile_t": tt, "sort_every": k, "ms_per_step": ms})
    ok = [t for t in table if t["ms_per_step"] is not None]
    best = min(ok, key=lambda t: t["ms_per_step"])
    return {"workload": workload, "grid": grid, "pairs": base["n_pairs"], "best": best, "table": table}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c3")
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--pairs", type=int, default=0)
    ap.add_argument("--steps", type=int, default=16)
    args = ap.parse_args()
    print(json.dumps(tune(args.workload, args.grid, steps=args.steps, pairs=args.pairs)))


if __name__ == "__main__":
    main()
