"""Radial-slab decomposition of one run through the CUDA library: two gloo
processes share the GPU, each stepping its slab as an hff instance on its
local rows (stage groups through hff_step_stages, J-halo sums through
hff_fields / hff_set_field, particle migration through hff_particles /
hff_load_particles), exchanging on the host.  Neither process's kernels wait
on the other's: every exchange goes through the host.

After ten steps of the 96 x 80 hybrid workload (FP64, injection on), every
owned row of E and B must equal the single-domain library run to 1e-11
relative, and the union of the slabs' particles its particles (cells
identical, states within 1e-10)."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = ("E_r", "E_th", "E_ph", "B_r", "B_th", "B_ph")
HALF = {"E_r", "B_th", "B_ph"}
STEPS = 10


def _workload():
    from paper_2406_14512_gb300 import workloads
    cfg = workloads.config("small_hybrid")
    cfg.update(capacity=60000, sort_every=8, precision="fp64")
    return cfg, workloads.particles(cfg, n_pairs=3000, seed=21)


def _worker(rank, world, port, q):
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import __graft_entry__
        __graft_entry__.build()
        from paper_2406_14512_gb300 import hff, slabs
        cfg, ps = _workload()
        ref = hff.Sim(cfg)
        fields0 = {n: ref.get(n) for n in FIELDS}
        for s in range(2):
            ref.load(s, ps[s])
        plan = slabs.partition_rows(slabs.row_counts([p["cell"] for p in ps], cfg["nr"], cfg["nt"]), world,
                                    halo=8)
        lo, hi = plan.local(rank)
        eng = slabs.LibrarySlab(cfg, lo, hi, fields0)
        a, b = plan.owned(rank)
        for s in range(2):
            row = ps[s]["cell"] // cfg["nt"]
            m = (row >= a) & (row < b)
            eng.set_particles(s, {k: v[m] for k, v in ps[s].items()})
        run = slabs.SlabRun(eng, plan, rank, dist)
        run.step(STEPS)
        ref.step(STEPS)
        out = {"rank": rank, "plan": plan.faces, "fields": {}, "parts": [], "status": eng.sim.status()}
        for name in FIELDS:
            g, l = ref.get(name), eng.get(name)
            ha, hb = plan.owned_half(rank) if name in HALF else plan.owned(rank)
            out["fields"][name] = float(np.abs(l[ha - lo:hb - lo] - g[ha:hb]).max() / max(np.abs(g).max(), 1e-300))
        for s in range(2):
            out["parts"].append(eng.particles(s))
            if rank == 0:
                out.setdefault("ref", []).append(ref.particles(s))
        eng.close()
        ref.close()
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


def test_library_slabs_reproduce_the_single_domain_run():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29800 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted([q.get(timeout=900) for _ in ps], key=lambda d: d["rank"])
    for p in ps:
        p.join(timeout=120)
    for r in res:
        assert "error" not in r, r.get("error")
        assert r["status"] == 0
    for r in res:
        for name, err in r["fields"].items():
            assert err < 1e-11, (r["rank"], name, err)
    for s in range(2):
        ref = _canon(res[0]["ref"][s])
        got = _canon({k: np.concatenate([r["parts"][s][k] for r in res]) for k in res[0]["parts"][s]})
        assert len(got["cell"]) == len(ref["cell"]) > 0
        assert np.array_equal(got["cell"], ref["cell"])
        for k in ("xo", "yo"):
            assert np.abs(got[k] - ref[k]).max() < 1e-10, k
        for k in ("ur", "ut", "up", "w"):
            assert np.abs(got[k] - ref[k]).max() <= 1e-10 * max(1.0, np.abs(ref[k]).max()), k
