"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs, element by element.

Tolerances: FP32 fields and currents after one step within a relative L2 of
1e-5; particle cells bit-exact except where the FP64 position lies within
1e-5 cell of a face; offsets within 1e-5 cell after 10 steps.  The FP64
instantiation of the same kernels is held to 1e-10 (summation order of the
atomic deposit is the only difference from the oracle).
"""
import numpy as np
import pytest

from helpers import FIELDS6, michel_fields, particle_mismatches, rel_l2, shared_initial_state

pytestmark = pytest.mark.gpu

ST = dict(node=1, correct=2, push=4, faraday1=8, ampere=16, faraday2=32, inject=64, sort=128, all=255)
FIELD_STAGES = ST["node"] | ST["faraday1"] | ST["ampere"] | ST["correct"] | ST["faraday2"]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2406_14512_gb300 import hff, workloads
    return hff, workloads, oracle


def make(env, name, **kw):
    hff, workloads, oracle = env
    cfg = workloads.config(name)
    cfg.update(kw)
    return cfg, hff.Sim(cfg), oracle.Oracle(cfg)


@pytest.mark.parametrize("name,prec,tol,extra", [
    ("small_hybrid", "fp32", 1e-5, {}), ("small_rr", "fp32", 1e-5, {}), ("small_michel", "fp32", 1e-5, {}),
    ("small_hybrid", "fp64", 1e-11, {}),
    # the corrections-only return with the fourth-difference filter of E_r, E_th
    ("small_hybrid", "fp32", 1e-5, {"ff_delta_only": 1, "ff_filter": 1.0}),
    ("small_michel", "fp64", 1e-11, {"ff_delta_only": 1, "ff_filter": 0.5}),
    # the corrections-only return with the corrected field on the stellar row
    # (ff_delta_only 2), alone and with the filter sharing the J_PIC slots
    ("small_hybrid", "fp32", 1e-5, {"ff_delta_only": 2}), ("small_michel", "fp64", 1e-11, {"ff_delta_only": 2}),
    ("small_hybrid", "fp64", 1e-11, {"ff_delta_only": 2, "ff_filter": 1.0}),
    # the fused pass (field_pass 1) on one strip and four segments, and on
    # several strips and row segments (halo columns and warm-up rows
    # crossing block boundaries), with the filter on nine
    ("small_hybrid", "fp32", 1e-5, {"field_pass": 1}), ("small_hybrid", "fp64", 1e-11, {"field_pass": 1}),
    ("small_michel", "fp32", 1e-5, {"field_pass": 1}),
    ("small_fine", "fp64", 1e-11, {"field_pass": 1}), ("small_fine", "fp32", 1e-5, {"field_pass": 1}),
    ("c1", "fp64", 1e-11, {"field_pass": 1, "ff_delta_only": 1, "ff_filter": 1.0}),
    ("c1", "fp32", 1e-5, {"field_pass": 1, "ff_delta_only": 1, "ff_filter": 1.0}),
    # the four separate field kernels, explicitly (the cases above without
    # field_pass take them too: small grids)
    ("small_fine", "fp64", 1e-11, {"field_pass": 2})])
def test_field_step_parity(env, name, prec, tol, extra):
    """Psi, J_perp, Yee advance, blended current, renormalisation, star and
    absorber: one field-only step from identical smooth fields, through the
    four separate field kernels (field_pass 2, and the automatic choice on
    these small grids) or the fused field pass (field_pass 1)."""
    cfg, sim, ref = make(env, name, capacity=0, precision=prec, sort_every=0, **extra)
    shared_initial_state(sim, ref, seed=3)
    psi_g = sim.get("psi")  # FP64 prefix of the current B_r
    ref_psi = oracle_psi(ref)
    assert rel_l2(psi_g, ref_psi) < (1e-7 if prec == "fp32" else 1e-13)
    sim.step_stages(1, FIELD_STAGES)
    ref.step(1, FIELD_STAGES)
    for f in FIELDS6:
        assert rel_l2(sim.get(f), ref.get(f)) < tol, (f, rel_l2(sim.get(f), ref.get(f)))
    for f in ("jperp_r", "jperp_th", "jperp_ph"):
        assert rel_l2(sim.get(f), ref.get(f)) < 10 * tol, f


def test_split_monopole_field_step_parity(env):
    """The split monopole (Michel's solution reversed in the south, its
    current sheet on the equator, force-free everywhere): one field step of
    the FP32 CUDA path against the FP64 oracle from identical inputs.  The
    hemispheres are exact negatives, so B^2 = 0 on the equatorial nodes in
    both precisions and both codes skip them identically.  E_r and E_ph
    start at zero and are judged within the E vector."""
    hff, workloads, oracle = env
    cfg = workloads.config("small_michel")
    cfg.update(psi_break=[-1.0], f_break=[1.0], capacity=0, precision="fp32", sort_every=0)
    sim, ref = hff.Sim(cfg), oracle.Oracle(cfg)
    for k, v in michel_fields(cfg, split=True, real=np.float32).items():
        sim.set(k, v)
        ref.set(k, v.astype(np.float64))
    sim.step_stages(1, FIELD_STAGES)
    ref.step(1, FIELD_STAGES)
    for f in ("B_r", "B_th", "B_ph"):
        assert rel_l2(sim.get(f), ref.get(f)) < 1e-5, (f, rel_l2(sim.get(f), ref.get(f)))
    e_ref = np.concatenate([ref.get(f).ravel() for f in ("E_r", "E_th", "E_ph")])
    e_gpu = np.concatenate([sim.get(f).ravel() for f in ("E_r", "E_th", "E_ph")])
    assert rel_l2(e_gpu, e_ref) < 1e-5, rel_l2(e_gpu, e_ref)
    for f in ("E_r", "E_th", "E_ph"):
        d = np.linalg.norm(sim.get(f).astype(np.float64) - ref.get(f)) / np.linalg.norm(e_ref)
        assert d < 1e-5, (f, d)
    assert sim.status() == 0


def oracle_psi(ref):
    """Psi of the oracle's current B_r (its node pass, run on a copy)."""
    import oracle
    o2 = oracle.Oracle(ref.cfg)
    o2.set("B_r", ref.get("B_r"))
    o2.step(1, oracle.ST["node"])
    return o2.get("psi")


@pytest.mark.parametrize("name,prec,tol", [("small_pic", "fp64", 1e-10), ("small_hybrid", "fp32", 1e-5),
                                           ("small_rr", "fp32", 1e-5), ("small_fine", "fp32", 1e-5)])
def test_push_deposit_parity(env, name, prec, tol):
    """Gather, Boris + radiation reaction, move, kill rules and the
    charge-conserving deposit for one step in frozen fields."""
    hff, workloads, _ = env
    cfg, sim, ref = make(env, name, capacity=20000, precision=prec, sort_every=0, inject=False)
    shared_initial_state(sim, ref, seed=7)
    ps = workloads.particles(cfg, n_pairs=6000, seed=21)
    for s in range(2):
        sim.load(s, ps[s])
        ref.set_particles(s, ps[s])
    sim.step_stages(1, ST["node"] | ST["push"])
    ref.step(1, ST["node"] | ST["push"])
    for f in ("J_r", "J_th", "J_ph"):
        assert rel_l2(sim.get(f), ref.get(f)) < tol, (f, rel_l2(sim.get(f), ref.get(f)))
    for s in range(2):
        g, o = sim.particles(s), ref.particles(s)
        bad, ties, err = particle_mismatches(g, o, cfg["nt"])
        assert bad == 0, (s, bad, ties)
        assert err < (1e-5 if prec == "fp32" else 1e-11), err
        live = (g["cell"] >= 0) & (g["cell"] == o["cell"])
        for k in ("ur", "ut", "up"):
            assert rel_l2(g[k][live], o[k][live]) < tol, k


@pytest.mark.parametrize("case", ["scattered", "cluster", "cell_order"])
def test_tiled_deposit_parity(env, case):
    """One push/deposit step of the FP32 tiled kernel (shared-memory J with
    FP32 shared atomics, flushed once per grid point) against the FP64
    oracle: J within 1e-6 in relative L2 (measured 1.2e-7 to 2.8e-7), and
    within 2e-6 with a third of the electrons, all with one momentum, piled
    into one cell (measured up to 1.1e-6), which after the tile sort sit
    next to each other, so that the deposit sums runs of equal windows
    within the warp before its atomics; likewise with every particle in cell
    order; particles as in the tail-kernel test.  (An int32 fixed-point
    shared J, about 2^-21 of the largest contribution per unit, measured
    1.7e-6 to 8.7e-6 here, and 1.45e-2 with a dense cell of mixed
    momenta.)"""
    hff, workloads, _ = env
    cfg, sim, ref = make(env, "small_hybrid", capacity=40000, precision="fp32", sort_every=4, inject=False)
    shared_initial_state(sim, ref, seed=7)
    ps = workloads.particles(cfg, n_pairs=8000, seed=23)
    if case == "cluster":
        e = ps[0]
        e["cell"][::3] = int(e["cell"][0])
        e["ur"][::3], e["ut"][::3], e["up"][::3] = 0.3, -0.2, 0.5
    if case == "cell_order":
        for s in range(2):
            o = np.argsort(ps[s]["cell"], kind="stable")
            ps[s] = {k: v[o] for k, v in ps[s].items()}
    cluster = case == "cluster"
    for s in range(2):
        sim.load(s, ps[s])
        ref.set_particles(s, ps[s])
    ref.sort_now()  # the GPU loader sorts; sort the oracle identically
    sim.step_stages(1, ST["node"] | ST["push"])
    ref.step(1, ST["node"] | ST["push"])
    assert sim.info().pushed_tiled > 0
    tol = 2e-6 if cluster else 1e-6
    for f in ("J_r", "J_th", "J_ph"):
        assert rel_l2(sim.get(f), ref.get(f)) < tol, (f, rel_l2(sim.get(f), ref.get(f)))
    for s in range(2):
        g, o = sim.particles(s), ref.particles(s)
        bad, ties, err = particle_mismatches(g, o, cfg["nt"])
        assert bad == 0, (s, bad, ties)
        assert err < 1e-5, err
    assert sim.status() == 0


def test_gauss_law_fp32_dense_cell(env):
    """A third of the pairs piled into one cell (each pair co-located, so
    the start is neutral), electrons with one momentum and positrons with the
    opposite one, so that their currents add in that cell's shared J: the
    FP32 graph path (tiled push, sorts every 4 steps) keeps the Gauss
    residual within 2e-5 of the charge density after 20 steps (measured
    4.3e-6; an int32 fixed-point shared J measured 3.3e-4), no flag raised."""
    hff, workloads, _ = env
    cfg, sim, ref = make(env, "small_pic", capacity=40000, precision="fp32", sort_every=4)
    ps = workloads.particles(cfg, n_pairs=5000, seed=61)
    c0 = int(ps[0]["cell"][0])
    for s, sign in ((0, 1.0), (1, -1.0)):
        ps[s]["cell"][::3] = c0
        ps[s]["ur"][::3], ps[s]["ut"][::3], ps[s]["up"][::3] = 0.3 * sign, -0.2 * sign, 0.5 * sign
    for s in range(2):
        sim.load(s, ps[s])
    sim.step(20)
    d, _ = sim.diagnostics()
    assert sim.info().pushed_tiled > 0
    assert d.rho_max > 0 and d.gauss_max < 2e-5 * d.rho_max, (d.gauss_max, d.rho_max)
    assert sim.status() == 0


@pytest.mark.parametrize("name,prec,extra", [
    ("small_pic", "fp64", {}), ("small_hybrid", "fp32", {}), ("small_rr", "fp32", {}), ("small_fine", "fp32", {}),
    # reading 2 of the field return (the stellar row takes the corrected field)
    ("small_hybrid", "fp64", {"ff_delta_only": 2}), ("small_hybrid", "fp32", {"ff_delta_only": 2})])
def test_ten_full_steps(env, name, prec, extra):
    """Ten whole steps (graph path: tiled push, injection, sort every 4):
    particle order and cells identical up to face ties and positions within
    1e-5 cell.  Fields: FP64 to 1e-10; FP32 to 1e-5 in relative L2 per
    field, the single-step tolerance, after all ten steps (measured: at most
    8e-7, E_ph of the finer grid)."""
    hff, workloads, _ = env
    cfg, sim, ref = make(env, name, capacity=60000, precision=prec, sort_every=4, **extra)
    ps = workloads.particles(cfg, n_pairs=8000, seed=31)
    for s in range(2):
        sim.load(s, ps[s])
        ref.set_particles(s, ps[s])
    ref.sort_now()  # the GPU loader sorts; sort the oracle identically
    sim.step(10)
    ref.step(10)
    assert sim.info().step == 10
    for s in range(2):
        g, o = sim.particles(s), ref.particles(s)
        bad, ties, err = particle_mismatches(g, o, cfg["nt"])
        assert bad == 0 and ties <= max(2, len(o["cell"]) // 2000), (s, bad, ties)
        assert err < 1e-5, err
    tol = 1e-5 if prec == "fp32" else 1e-10
    errs = {f: rel_l2(sim.get(f), ref.get(f)) for f in FIELDS6}
    assert max(errs.values()) < tol, errs
    assert sim.status() == 0


def test_sort_bit_exact(env):
    """Stable tile sort with compaction: identical order to the oracle's
    stable counting sort (ties keep their prior order)."""
    hff, workloads, _ = env
    cfg, sim, ref = make(env, "small_hybrid", capacity=30000, sort_every=1, tile_r=8, tile_t=16, inject=False)
    ps = workloads.particles(cfg, n_pairs=9000, seed=41)
    for s in range(2):
        p = {k: v.copy() for k, v in ps[s].items()}
        p["cell"][::5] = -1
        sim.load(s, p)  # sorts on load
        ref.set_particles(s, p)
    ref.step(1, ST["sort"])
    for s in range(2):
        g, o = sim.particles(s), ref.particles(s)
        assert np.array_equal(g["cell"], o["cell"])
        assert np.array_equal(g["xo"].astype(np.float64), o["xo"])
        assert np.array_equal(g["w"].astype(np.float64), o["w"])


def test_injection_bit_exact(env):
    """Top-up injection: counts, cells and offsets identical to the oracle
    (Philox4x32-10 on both sides, keyed by seed, step, cell, k)."""
    hff, workloads, oracle = env
    for prec in ("fp64", "fp32"):
        cfg, sim, ref = make(env, "small_pic", capacity=50000, sort_every=0, precision=prec)
        sim.step_stages(1, ST["inject"])
        ref.step(1, ST["inject"])
        for s in range(2):
            g, o = sim.particles(s), ref.particles(s)
            assert len(g["cell"]) == len(o["cell"]) > 0
            assert np.array_equal(g["cell"], o["cell"])
            assert np.array_equal(g["xo"].astype(np.float64), o["xo"])
            assert np.array_equal(g["yo"].astype(np.float64), o["yo"])
            assert np.allclose(g["up"], o["up"], rtol=1e-6 if prec == "fp32" else 1e-14, atol=0)
            assert np.all(g["ur"] == 0) and np.all(g["ut"] == 0)
        # later steps: the deficit follows the surface counts after each move.
        # Which particles end a push in a surface cell is decided in floating
        # point, whose rounding order differs between the two codes, so the
        # free-running counts may differ by a particle at a cell face (loose
        # check at the end).  The injection itself is checked exactly: the
        # oracle injects from the GPU's own pushed state and surface counts.
        for n in range(3):
            sim.step_stages(1, ST["node"] | ST["push"] | hff.ST["nocount"])
            ref.step(1, ST["node"] | ST["push"] | ST["inject"])
            pre = [sim.particles(s) for s in range(2)]
            chk = oracle.Oracle(cfg)
            surf = np.zeros(cfg["nt"], np.int64)
            for s in range(2):
                chk.set_particles(s, pre[s])
                c = pre[s]["cell"]
                surf += np.bincount(c[(c >= 0) & (c < cfg["nt"])], minlength=cfg["nt"])
            chk.set_surface_counts(surf)
            chk.step_index = sim.info().step
            sim.step_stages(1, ST["inject"])
            chk.step(1, ST["inject"])
            for s in range(2):
                g, o = sim.particles(s), chk.particles(s)
                assert len(g["cell"]) == len(o["cell"]) > len(pre[s]["cell"]), (n, s)
                assert np.array_equal(g["cell"], o["cell"])
                assert np.array_equal(g["xo"].astype(np.float64), o["xo"])
                assert np.array_equal(g["yo"].astype(np.float64), o["yo"])
                k = len(pre[s]["cell"])
                assert np.allclose(g["up"][k:], o["up"][k:], rtol=1e-6 if prec == "fp32" else 1e-14, atol=0)
        for s in range(2):
            assert abs(len(sim.particles(s)["cell"]) - ref.count(s)) <= 2


def test_diagnostics_parity(env):
    hff, workloads, _ = env
    cfg, sim, ref = make(env, "small_pic", capacity=40000, precision="fp64", sort_every=4)
    ps = workloads.particles(cfg, n_pairs=5000, seed=51)
    for s in range(2):
        sim.load(s, ps[s])
        ref.set_particles(s, ps[s])
    ref.sort_now()
    sim.step(8)
    ref.step(8)
    dg, pg = sim.diagnostics()
    do, po = ref.diagnostics()
    assert rel_l2(pg, po) < 1e-9
    for k in ("psi_open", "u_e", "u_b", "rho_max", "injected", "killed"):
        a, b = getattr(dg, k), getattr(do, k)
        assert abs(a - b) <= 1e-9 * max(abs(b), 1e-30), (k, a, b)
    assert abs(dg.radiated - do.radiated) <= 1e-9 * max(abs(do.radiated), 1e-30)
    for s in range(2):
        assert dg.count[s] == do.count[s]
        assert abs(dg.kinetic[s] - do.kinetic[s]) <= 1e-9 * do.kinetic[s]
    # Gauss's law: both at round-off of FP64
    assert dg.gauss_max < 1e-9 * dg.rho_max and do.gauss_max < 1e-9 * do.rho_max


def test_gauss_law_fp32_graph(env):
    """Charge-conserving deposit in FP32 through the graph path: the Gauss
    residual stays at FP32 round-off relative to the charge density, within
    1e-6 after 20 steps (measured 1.3e-7 to 1.7e-7, the same as the untiled
    push; an int32 fixed-point shared J measured 5.8e-5)."""
    hff, workloads, _ = env
    cfg, sim, ref = make(env, "small_pic", capacity=40000, precision="fp32", sort_every=4)
    ps = workloads.particles(cfg, n_pairs=5000, seed=61)
    for s in range(2):
        sim.load(s, ps[s])
    sim.step(20)
    d, _ = sim.diagnostics()
    assert d.rho_max > 0 and d.gauss_max < 1e-6 * d.rho_max, (d.gauss_max, d.rho_max)
