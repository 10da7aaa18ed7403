"""Threshold pair creation (Sect. 5.1) through the C ABI against the oracle.

The push records an event for every lepton above gamma_th; after the
injection the pairs are appended in parent order, so the particle arrays
stay index-aligned with the oracle's.  The threshold test is a floating-point
decision: the inputs are checked to keep every lepton at least 1e-4 (relative,
in gamma^2) away from it, far beyond the FP32/FP64 difference of a push."""
import numpy as np
import pytest

from helpers import FIELDS6, particle_mismatches, rel_l2

pytestmark = pytest.mark.gpu


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


def setup(env, precision, sort_every, seed=21, **kw):
    hff, workloads, oracle = env
    cfg = workloads.config("small_pairs")
    cfg.update(precision=precision, sort_every=sort_every, capacity=80000, **kw)
    ps = workloads.particles(cfg, seed=seed)
    sim, ref = hff.Sim(cfg), oracle.Oracle(cfg)
    for s in range(2):
        sim.load(s, ps[s])
        ref.set_particles(s, ps[s])
    if sort_every:
        ref.sort_now()
    return cfg, sim, ref


def margin_ok(ref, cfg, n):
    """Every live lepton of the first n slots is clear of the threshold."""
    g2 = cfg["gamma_th"] ** 2
    for s in range(2):
        p = ref.particles(s)
        u2 = p["ur"][:n[s]] ** 2 + p["ut"][:n[s]] ** 2 + p["up"][:n[s]] ** 2
        live = p["cell"][:n[s]] >= 0
        if live.any() and np.min(np.abs(1.0 + u2[live] - g2)) < 1e-4 * g2:
            return False
    return True


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
def test_one_step_with_pair_creation(env, precision, tol):
    cfg, sim, ref = setup(env, precision, sort_every=0)
    n0 = [ref.count(0), ref.count(1)]
    sim.step(1)
    ref.step(1)
    assert margin_ok(ref, cfg, n0)
    dr, dg = ref.diagnostics()[0], sim.diagnostics()[0]
    assert dr.created > 0
    assert abs(dg.created - dr.created) <= 1e-5 * dr.created
    assert sim.info().count[0] == ref.count(0) and sim.info().count[1] == ref.count(1)
    for s in range(2):
        g, o = sim.particles(s), ref.particles(s)
        bad, ties, err = particle_mismatches(g, o, cfg["nt"])
        assert bad == 0 and ties <= 2, (s, bad, ties)
        assert err < 1e-5
        live = (g["cell"] >= 0) & (g["cell"] == o["cell"])
        for k in ("ur", "ut", "up", "w"):
            assert rel_l2(g[k][live], o[k][live]) < 10 * tol, k
    errs = {f: rel_l2(sim.get(f), ref.get(f)) for f in FIELDS6}
    assert max(errs.values()) < tol, errs
    assert sim.status() == 0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_ten_steps_with_pair_creation_and_sorting(env, precision):
    """Radiation reaction off: the leptons above the threshold stay there
    (no cooling through gamma_th, where FP32 and FP64 could decide apart),
    and create a pair every step; the margin is checked at every step."""
    cfg, sim, ref = setup(env, precision, sort_every=4, seed=23, gamma_rad=0.0)
    sim.step(10)
    for _ in range(10):
        n = [ref.count(0), ref.count(1)]
        ref.step(1)
        assert margin_ok(ref, cfg, n)
    assert ref.diagnostics()[0].created > 0
    for s in range(2):
        g, o = sim.particles(s), ref.particles(s)
        bad, ties, err = particle_mismatches(g, o, cfg["nt"])
        assert bad == 0 and ties <= max(2, len(o["cell"]) // 2000), (s, bad, ties)
        assert err < 1e-5, err
    tol = 1e-5 if precision == "fp32" else 1e-10
    errs = {f: rel_l2(sim.get(f), ref.get(f)) for f in FIELDS6}
    assert max(errs.values()) < tol, errs
    assert sim.status() == 0


@pytest.mark.parametrize("precision,steps", [("fp32", 1), ("fp64", 10)])
def test_crust_extraction_with_protons(env, precision, steps):
    """Three species (e-, e+, protons with m_p = 1836 m_e), electrons and
    protons injected from the surface (Sect. 5.1), pair creation and
    radiation reaction on, Table 1 flux bands.  FP64 over ten steps with
    sorting; FP32 over one step with the threshold margin checked."""
    hff, workloads, oracle = env
    cfg = workloads.config("small_crust")
    cfg.update(precision=precision, sort_every=4, capacity=80000)
    ps = workloads.particles(cfg, seed=25)
    sim, ref = hff.Sim(cfg), oracle.Oracle(cfg)
    for s in range(2):
        sim.load(s, ps[s])
        ref.set_particles(s, ps[s])
    ref.sort_now()
    sim.step(steps)
    for _ in range(steps):
        n = [ref.count(0), ref.count(1)]
        ref.step(1)
        if precision == "fp32":
            assert margin_ok(ref, cfg, n)
    d = ref.diagnostics()[0]
    assert d.count[2] > 0
    for s in range(3):
        g, o = sim.particles(s), ref.particles(s)
        bad, ties, err = particle_mismatches(g, o, cfg["nt"])
        assert bad == 0 and ties <= max(2, len(o["cell"]) // 2000), (s, bad, ties)
        assert err < 1e-5, err
    tol = 1e-5 if precision == "fp32" else 1e-10
    errs = {f: rel_l2(sim.get(f), ref.get(f)) for f in FIELDS6}
    assert max(errs.values()) < tol, errs
    assert sim.status() == 0
