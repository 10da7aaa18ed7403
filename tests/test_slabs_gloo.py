"""Radial-slab decomposition of one run (paper_2406_14512_gb300.slabs) against
the single-domain oracle: two (and three) gloo ranks on the CPU, each computing its slab
with an FP64 oracle built on its local rows, exchanging the J-halo sum, the E
and B halo rows and migrating particles, for ten whole steps of the hybrid
workload (Table 1 bands, injection, sorting in the reference run).

The owned rows of every field and the union of the ranks' particles must
equal the single-domain run.  Not bit for bit: a node's J is summed in another
order (each rank's own deposits, then its neighbour's), so the comparison is
at 1e-12 relative (fields) and 1e-10 of a cell (particles); cells and counts
are exact.
"""
import math
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = ("E_r", "E_th", "E_ph", "B_r", "B_th", "B_ph")
HALF = {"E_r", "B_th", "B_ph", "J_r", "B0_th", "B0_ph"}
STEPS = 10


def _workload():
    from paper_2406_14512_gb300 import workloads
    cfg = workloads.config("small_hybrid")
    cfg.update(capacity=60000, sort_every=8)
    return cfg, workloads.particles(cfg, n_pairs=3000, seed=21)


class OracleSlab:
    """A slab of the run computed by the FP64 oracle on node rows lo .. hi."""

    def __init__(self, oracle, cfg, lo, hi, ref):
        d = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["nr"]
        r_lo, r_hi = cfg["r_min"] * math.exp(lo * d), cfg["r_min"] * math.exp(hi * d)
        # the oracle's absorber ramps to its own r_max: a slab that stops short
        # of the outer edge must lie wholly inside r_abs
        assert hi == cfg["nr"] or r_hi <= cfg["r_abs"], "slab reaches into the absorber"
        c = dict(cfg, nr=hi - lo, r_min=r_lo, r_max=r_hi, inject=bool(cfg["inject"]) and lo == 0)
        # same magnetic moment (flux unit) and the same time step as the whole run
        c["b_star"] = cfg["b_star"] * (cfg["r_min"] / r_lo) ** 3
        dt = oracle.config_dt(cfg)
        c["courant"] = dt / oracle.config_dt(dict(c, courant=1.0))
        self.o = oracle.Oracle(c)
        assert abs(self.o.dt / dt - 1) < 1e-14
        self.lo, self.hi, self.nt, self.n_species = lo, hi, cfg["nt"], self.o.n_species
        for name in FIELDS + ("B0_r", "B0_th", "B0_ph"):
            a = ref.get(name)
            self.o.set(name, a[lo:hi if name in HALF else hi + 1])
        self.o.step_index = ref.step_index

    def stages(self, mask):
        k = self.o.step_index
        self.o.step(1, mask)
        self.o.step_index = k

    def count_step(self):
        self.o.step_index = self.o.step_index + 1

    def get(self, name):
        return self.o.get(name)

    def set(self, name, a):
        self.o.set(name, a)

    def particles(self, s):
        p = self.o.particles(s)
        p["cell"] = np.where(p["cell"] >= 0, p["cell"] + self.lo * self.nt, -1).astype(np.int32)
        return p

    def set_particles(self, s, p):
        q = dict(p)
        q["cell"] = np.where(p["cell"] >= 0, p["cell"] - self.lo * self.nt, -1).astype(np.int32)
        self.o.set_particles(s, q)


def _worker(rank, world, port, q):
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import oracle
        from paper_2406_14512_gb300 import slabs
        cfg, ps = _workload()
        ref = oracle.Oracle(cfg)
        for s in range(2):
            ref.set_particles(s, ps[s])
        plan = slabs.partition_rows(slabs.row_counts([p["cell"] for p in ps], cfg["nr"], cfg["nt"]), world,
                                    halo=8)
        lo, hi = plan.local(rank)
        eng = OracleSlab(oracle, cfg, lo, hi, ref)
        a, b = plan.owned(rank)
        for s in range(2):
            row = ps[s]["cell"] // cfg["nt"]
            m = (row >= a) & (row < b)
            eng.set_particles(s, {k: v[m] for k, v in ps[s].items()})
        run = slabs.SlabRun(eng, plan, rank, dist)
        run.step(STEPS)
        ref.step(STEPS)
        out = {"rank": rank, "plan": plan.faces, "fields": {}, "parts": []}
        for name in FIELDS:
            g, l = ref.get(name), eng.get(name)
            ha, hb = plan.owned_half(rank) if name in HALF else plan.owned(rank)
            err = np.abs(l[ha - lo:hb - lo] - g[ha:hb]).max() / max(np.abs(g).max(), 1e-300)
            out["fields"][name] = float(err)
        for s in range(2):
            out["parts"].append(eng.particles(s))
            if rank == 0:
                out.setdefault("ref", []).append(ref.particles(s))
        q.put(out)
        dist.destroy_process_group()
    except Exception as ex:  # report instead of hanging the parent
        import traceback
        q.put({"rank": rank, "error": traceback.format_exc() + str(ex)})


def _canon(p):
    live = p["cell"] >= 0
    keys = ("cell", "xo", "yo", "ur", "ut", "up", "w")
    a = {k: np.asarray(p[k])[live] for k in keys}
    order = np.lexsort((a["yo"], a["xo"], a["cell"]))
    return {k: v[order] for k, v in a.items()}


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_reproduce_the_single_domain_run(world):
    """Two ranks (one face), and three (a middle rank with two neighbours)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + (os.getpid() * 7 + world) % 1000
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted([q.get(timeout=600) for _ in ps], key=lambda d: d["rank"])
    for p in ps:
        p.join(timeout=60)
    for r in res:
        assert "error" not in r, r.get("error")
    faces = res[0]["plan"]
    assert len(faces) == world + 1 and all(faces[k] < faces[k + 1] for k in range(world))
    for r in res:
        for name, err in r["fields"].items():
            assert err < 1e-12, (r["rank"], name, err)
    for s in range(2):
        ref = _canon(res[0]["ref"][s])
        got = _canon({k: np.concatenate([r["parts"][s][k] for r in res]) for k in res[0]["parts"][s]})
        assert len(got["cell"]) == len(ref["cell"]) > 0
        assert np.array_equal(got["cell"], ref["cell"])
        for k in ("xo", "yo"):
            assert np.abs(got[k] - ref[k]).max() < 1e-10, k
        for k in ("ur", "ut", "up", "w"):
            assert np.abs(got[k] - ref[k]).max() <= 1e-10 * max(1.0, np.abs(ref[k]).max()), k


def test_partition_balances_particles_and_keeps_slabs_wide():
    from paper_2406_14512_gb300 import slabs
    counts = np.zeros(100, np.int64)
    counts[60:70] = 1000          # a dense sheet far out
    counts[:60] = 10
    plan = slabs.partition_rows(counts, 2, halo=6)
    a = counts[:plan.faces[1]].sum()
    assert abs(a - counts.sum() / 2) <= 1000
    plan4 = slabs.partition_rows(counts, 4, halo=6)
    widths = np.diff(plan4.faces)
    assert widths.min() >= 11 and plan4.faces[-1] == 100
    with pytest.raises(ValueError):
        slabs.partition_rows(counts, 10, halo=6)
    with pytest.raises(ValueError):
        slabs.partition_rows(counts, 2, halo=3)
