"""Autotuner of the launch shape: tile size of the particle sort (and of the
tiled push's shared-memory region) and the sort cadence.

Two entry points:
  * resolve(cfg, particles) -- the init path.  A configuration whose tile_r,
    tile_t are 0 and sort_every is AUTO asks for its launch shape to be
    measured: every candidate is timed on a throwaway instance of the very
    configuration and particles that will run (whole graph-replayed steps,
    sorts included), the fastest is written into the configuration, and the
    choice is cached per device, grid, precision and particle count, so the
    probe runs once.  Without particles the cached choice, else DEFAULT_SHAPE,
    is used.  hff.Sim(cfg, particles=...) calls it.
  * tune(workload, grid) -- the same timing on an n x n sample of a named
    workload (same particles per cell), for exploring shapes offline.
The tile with its halo must fit the shared memory of one block, so large
tiles are only tried with short cadences.  GPU only: the timings are CUDA
events around graph-replayed steps.

    python -m paper_2406_14512_gb300.autotune --workload c3 --grid 1024
"""
from __future__ import annotations

import argparse
import json
import itertools
import os

DEFAULT_TILES = [(8, 32), (16, 16), (16, 24), (16, 32), (32, 32)]
DEFAULT_CADENCES = [4, 8, 12, 16]
AUTO = -1                      # sort_every value that asks for the autotuner
INIT_TILES = [(16, 16), (16, 24), (16, 32), (32, 16)]
INIT_CADENCES = [8, 12, 16]
DEFAULT_SHAPE = (16, 24, 12)   # fallback when nothing was measured
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune_cache.json")


def wants_tuning(cfg: dict) -> bool:
    return (int(cfg.get("tile_r", 16)) == 0 and int(cfg.get("tile_t", 32)) == 0
            and int(cfg.get("sort_every", 0)) == AUTO)


def _key(cfg: dict, n_particles: int) -> str:
    import torch
    dev = torch.cuda.get_device_name(torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"
    n = int(float(f"{max(n_particles, 1):.2g}"))  # two significant digits
    return (f"{dev}|{cfg['nr']}x{cfg['nt']}|r{cfg['r_min']:g}-{cfg['r_max']:g}|lc{cfg['r_lc']:g}|"
            f"{cfg.get('precision', 'fp32')}|n{n}|rr{int(cfg.get('gamma_rad', 0) > 0)}")


def _cache_read() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _cache_write(d: dict) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, CACHE)


def resolve(cfg: dict, particles=None, tiles=None, cadences=None, steps: int = 48, warmup: int = 3,
            use_cache: bool = True) -> dict:
    """The configuration with its launch shape filled in (see the module
    docstring).  A configuration that does not ask for tuning is returned
    unchanged.  The result carries the probe table under "autotune".  The
    timed window (48 steps) is a multiple of every default cadence, so that
    each candidate is charged its exact share of sorts."""
    if not wants_tuning(cfg):
        return cfg
    n = 0 if particles is None else sum(len(p["cell"]) for p in particles)
    key = _key(cfg, n)
    cache = _cache_read() if use_cache else {}
    out = dict(cfg)
    if key in cache:
        hit = cache[key]
        out.update(tile_r=hit["tile_r"], tile_t=hit["tile_t"], sort_every=hit["sort_every"])
        out["autotune"] = {"source": "cache", "key": key, **hit}
        return out
    if particles is None:
        out.update(tile_r=DEFAULT_SHAPE[0], tile_t=DEFAULT_SHAPE[1], sort_every=DEFAULT_SHAPE[2])
        out["autotune"] = {"source": "default (no particles to measure with)", "key": key}
        return out
    from . import hff
    table = []
    for (tr, tt), k in itertools.product(tiles or INIT_TILES, cadences or INIT_CADENCES):
        c = dict(cfg, tile_r=tr, tile_t=tt, sort_every=k)
        try:
            ms = time_candidate(c, particles, steps, warmup)
        except hff.HffError as e:
            table.append({"tile_r": tr, "tile_t": tt, "sort_every": k, "ms_per_step": None, "error": str(e)})
            continue
        table.append({"tile_r": tr, "tile_t": tt, "sort_every": k, "ms_per_step": ms})
    ok = [t for t in table if t["ms_per_step"] is not None]
    if not ok:
        raise hff.HffError(hff.HFF_ERR_ARG, "no candidate launch shape fits this configuration")
    best = min(ok, key=lambda t: t["ms_per_step"])
    choice = {"tile_r": best["tile_r"], "tile_t": best["tile_t"], "sort_every": best["sort_every"],
              "ms_per_step": best["ms_per_step"]}
    if use_cache:
        cache = _cache_read()
        cache[key] = choice
        _cache_write(cache)
    out.update(tile_r=best["tile_r"], tile_t=best["tile_t"], sort_every=best["sort_every"])
    out["autotune"] = {"source": "measured", "key": key, **choice, "table": table}
    return out


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
