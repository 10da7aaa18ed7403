"""The 8192 x 8192, 1e9-particle precision-stress workload (r in [1, 200],
R_LC = 20): the largest grid and particle count the path supports in one
instance, where a cell index reaches 6.7e7 and each species holds 5e8
particles.

* The particles that start in a band of rows are pushed by the oracle; their
  current on the band's inner rows and their new states must agree with the
  GPU's (FP32), as in the 4096^2 test, so that no index product overflows.
* The FP32 and FP64 instantiations of the same kernels take one whole step
  from the same inputs: every field within the single-step tolerance
  (relative L2 1e-5), particle cells identical except at face ties, offsets
  within 1e-5 cell, and the FP64 flux function of both within 1e-6.
  E_ph is held to 1e-5 of |E|: it starts at zero, and after one step it is
  the sum of near-cancelling terms (the curl of a nearly curl-free B, and
  the J_ph of co-located injected e+- pairs, equal and opposite up to the
  rounding of the FP32 deposit), so its own relative error says nothing
  about the precision of E.

Device memory: one instance at a time (FP32 about 90 GB, FP64 about 150 GB)."""
import gc

import numpy as np
import pytest

from helpers import FIELDS6, particle_mismatches, rel_l2

pytestmark = pytest.mark.gpu

ST = dict(node=1, correct=2, push=4, faraday1=8, ampere=16, faraday2=32, inject=64, sort=128, all=255)


def host_available() -> float:
    """MemAvailable of /proc/meminfo in bytes (0 if unreadable)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return float(line.split()[1]) * 1024
    except OSError:
        pass
    return 0.0


@pytest.fixture(scope="module")
def c4():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    free_dev, total_dev = torch.cuda.mem_get_info()
    short = None
    if free_dev < 170e9:
        short = f"needs 170 GB of free device memory, {free_dev / 1e9:.0f} GB free"
    elif host_available() < 120e9:
        short = f"needs 120 GB of available host memory, {host_available() / 1e9:.0f} GB available"
    if short:
        # on a GPU whose memory could hold the workload, missing room is a
        # failure (the precision-stress workload must not drop out of a run
        # unnoticed); smaller GPUs, or an explicit opt-out, skip
        if total_dev >= 200e9 and os.environ.get("HFF_ALLOW_C4_SKIP") != "1":
            pytest.fail(short + " (set HFF_ALLOW_C4_SKIP=1 to skip)")
        pytest.skip(short)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_14512_gb300 import hff, workloads
    cfg = workloads.config("c4")
    cfg["capacity"] = int(cfg["n_pairs"] * 1.02) + 100_000
    ps = workloads.particles(cfg, threads=16)
    return hff, cfg, ps


def free(sim):
    import torch
    sim.close()
    del sim.mem
    gc.collect()
    torch.cuda.empty_cache()


def test_c4_band_push_deposit(c4):
    import oracle
    hff, cfg, ps = c4
    nt = cfg["nt"]
    sim = hff.Sim(cfg)
    cfg = sim.cfg  # the launch shape the autotuner resolved
    for s in range(2):
        sim.load(s, ps[s])
    lo, hi = 3560, 3576                 # rows near r = R_LC / 2 (dipole zone, PIC band)
    base = {}
    sel = {}
    for s in range(2):
        v = sim.particle_views(s)
        row = v["cell"] // nt
        idx = ((row >= lo) & (row <= hi)).nonzero().flatten()
        sel[s] = idx.cpu().numpy()
        base[s] = {k: t[idx].cpu().numpy() for k, t in v.items()}
    assert len(sel[0]) > 10_000
    ref = oracle.Oracle(dict(cfg, capacity=2 * max(len(sel[0]), len(sel[1])) + 1000, inject=False))
    for s in range(2):
        ref.set_particles(s, base[s])
    sim.step_stages(1, ST["node"] | ST["push"])
    ref.step(1, ST["node"] | ST["push"])
    a, b = lo + 2, hi
    for f in ("J_r", "J_th", "J_ph"):
        gj, oj = sim.get(f)[a:b], ref.get(f)[a:b]
        assert rel_l2(gj, oj) < 1e-5, (f, rel_l2(gj, oj))
    import torch
    for s in range(2):
        v = sim.particle_views(s)
        idx = torch.from_numpy(sel[s]).to(v["cell"].device)
        g = {k: t[idx].cpu().numpy() for k, t in v.items()}
        o = ref.particles(s)
        bad, ties, err = particle_mismatches(g, o, nt)
        assert bad == 0, (s, bad, ties)
        assert err < 1e-5
    assert sim.status() == 0
    free(sim)


def run_steps(hff, cfg, ps, precision, nsteps=1, stride=997):
    import torch
    sim = hff.Sim(dict(cfg, precision=precision))
    for s in range(2):
        sim.load(s, ps[s])
    sim.step(nsteps)
    out = {"fields": {f: sim.get(f) for f in FIELDS6}, "psi": sim.get("psi"), "parts": []}
    for s in range(2):
        v = sim.particle_views(s)
        out["parts"].append({k: t[::stride].to(torch.float64 if k != "cell" else torch.int32).cpu().numpy()
                             for k, t in v.items()})
    out["status"] = sim.status()
    out["info"] = sim.info()
    free(sim)
    return out


def test_c4_fp32_vs_fp64(c4):
    hff, cfg, ps = c4
    r32 = run_steps(hff, cfg, ps, "fp32")
    r64 = run_steps(hff, cfg, ps, "fp64")
    assert r32["status"] == 0 and r64["status"] == 0
    assert r32["info"].count[0] == r64["info"].count[0]
    f32, f64 = r32["fields"], r64["fields"]
    for f in ("E_r", "E_th", "B_r", "B_th", "B_ph"):
        assert rel_l2(f32[f], f64[f]) < 1e-5, (f, rel_l2(f32[f], f64[f]))
    e_norm = np.sqrt(sum(np.linalg.norm(f64[f].astype(np.float64)) ** 2 for f in ("E_r", "E_th", "E_ph")))
    d_ph = np.linalg.norm(f32["E_ph"].astype(np.float64) - f64["E_ph"])
    assert d_ph < 1e-5 * e_norm, d_ph / e_norm
    assert rel_l2(r32["psi"], r64["psi"]) < 1e-6
    for s in range(2):
        bad, ties, err = particle_mismatches(r32["parts"][s], r64["parts"][s], cfg["nt"])
        n = len(r64["parts"][s]["cell"])
        assert bad == 0 and ties <= max(2, n // 2000), (s, bad, ties)
        assert err < 1e-5, err
