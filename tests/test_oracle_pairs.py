"""Pins of the oracle's threshold pair creation (Sect. 5.1): a lepton whose
Lorentz factor after its push exceeds gamma_th creates one e- and one e+ at
its position, moving along its direction of motion with Lorentz factor
gamma_s; the parent is kept (reading).  The pairs are appended after the
injected particles in parent order: species 0 by slot, then species 1."""
import math

import numpy as np

from paper_2406_14512_gb300 import workloads

ST = dict(node=1, correct=2, push=4, faraday1=8, ampere=16, faraday2=32, inject=64, sort=128, all=255)


def pairs_cfg(**kw):
    cfg = workloads.config("small_pairs")
    cfg.update(precision="fp64", capacity=60000, sort_every=0, inject=False)
    cfg.update(kw)
    return cfg


def loaded(oracle_mod, cfg, seed=5, n=4000):
    o = oracle_mod.Oracle(cfg)
    ps = workloads.particles(cfg, n_pairs=n, seed=seed)
    for s in range(2):
        o.set_particles(s, ps[s])
    return o


def test_pairs_follow_the_threshold_rule(oracle_mod):
    cfg = pairs_cfg()
    o = loaded(oracle_mod, cfg)
    n0 = [o.count(0), o.count(1)]
    o.step(1, ST["all"] & ~ST["sort"])
    parts = [o.particles(s) for s in range(2)]
    gth2, us = cfg["gamma_th"] ** 2, math.sqrt(cfg["gamma_s"] ** 2 - 1.0)
    parents = []
    for s in range(2):
        p = parts[s]
        u2 = p["ur"][:n0[s]] ** 2 + p["ut"][:n0[s]] ** 2 + p["up"][:n0[s]] ** 2
        live = p["cell"][:n0[s]] >= 0
        parents += [(s, k) for k in np.flatnonzero(live & (1.0 + u2 > gth2))]
    assert len(parents) > 20                      # the inputs do reach the threshold
    wsum = 0.0
    for s in range(2):
        assert o.count(s) - n0[s] == len(parents)  # one particle of each species per parent
    for idx, (s, k) in enumerate(parents):
        par = {q: parts[s][q][k] for q in parts[s]}
        upar = np.array([par["ur"], par["ut"], par["up"]])
        wsum += par["w"]
        for sp in range(2):
            c = {q: parts[sp][q][n0[sp] + idx] for q in parts[sp]}
            assert c["cell"] == par["cell"] and c["xo"] == par["xo"] and c["yo"] == par["yo"]
            assert c["w"] == par["w"]
            uc = np.array([c["ur"], c["ut"], c["up"]])
            assert abs(np.linalg.norm(uc) - us) < 1e-12 * us
            # along the parent's direction of motion
            assert np.linalg.norm(np.cross(uc, upar)) < 1e-12 * us * np.linalg.norm(upar)
            assert uc @ upar > 0
    d, _ = o.diagnostics()
    assert abs(d.created - 2 * wsum) <= 1e-12 * 2 * wsum


def test_below_threshold_nothing_is_created(oracle_mod):
    """A threshold above every Lorentz factor in play creates nothing, and
    the run is then identical to one without pair creation."""
    a = loaded(oracle_mod, pairs_cfg(gamma_th=1e9))
    b = loaded(oracle_mod, pairs_cfg(gamma_th=0.0))
    a.step(3, ST["all"] & ~ST["sort"])
    b.step(3, ST["all"] & ~ST["sort"])
    for s in range(2):
        pa, pb = a.particles(s), b.particles(s)
        assert len(pa["cell"]) == len(pb["cell"])
        for q in pa:
            assert np.array_equal(pa[q], pb[q])
    assert a.diagnostics()[0].created == 0


def test_gauss_law_with_pair_creation(oracle_mod):
    """The created pairs are neutral and appear at one point, so the
    charge-conserving scheme keeps div E = 4 pi rho to round-off through
    creation, injection and sorting."""
    cfg = pairs_cfg(inject=True, sort_every=4, capacity=200000)
    o = loaded(oracle_mod, cfg, seed=9)
    for _ in range(3):
        o.step(5)
        d, _ = o.diagnostics()
        assert d.rho_max > 0
        assert d.gauss_max < 1e-9 * d.rho_max, (d.gauss_max, d.rho_max)
    assert d.created > 0


def test_crust_extraction_injects_electrons_and_protons(oracle_mod):
    """Sect. 5.1: the surface supplies electrons and protons (m_p = 1836 m_e)
    in corotation with no poloidal momentum, topping up each eligible cell to
    its target; with pair creation off the positron species gets nothing."""
    cfg = workloads.config("small_crust")
    cfg.update(precision="fp64", capacity=20000, sort_every=0, gamma_th=0.0)
    o = oracle_mod.Oracle(cfg)
    o.step(1, ST["inject"])
    tgt = o.inject_targets()
    assert tgt.sum() > 0
    e, pos, pr = (o.particles(s) for s in range(3))
    assert len(pos["cell"]) == 0
    assert len(e["cell"]) == len(pr["cell"]) == tgt.sum()
    for k in ("cell", "xo", "yo", "ur", "ut", "up", "w"):
        assert np.array_equal(e[k], pr[k]), k           # co-located: neutral at birth
    assert not e["ur"].any() and not e["ut"].any()
    # corotation: u_phi = gamma v, v = Omega r sin(theta) at the particle
    nt = cfg["nt"]
    d = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["nr"]
    r = cfg["r_min"] * np.exp(e["xo"] * d)
    th = (e["cell"] % nt + e["yo"]) * math.pi / nt
    v = r * np.sin(th) / cfg["r_lc"]
    assert np.allclose(e["up"], v / np.sqrt(1 - v * v), rtol=1e-14, atol=0)
    # per-cell counts equal the targets (first injection: no plasma yet)
    assert np.array_equal(np.bincount(e["cell"], minlength=nt)[:nt], tgt)


def test_crust_run_keeps_gauss_law_with_three_species(oracle_mod):
    """e-, e+ and protons with injection, pair creation and radiation
    reaction: Gauss's law to round-off in the PIC domain."""
    cfg = workloads.config("small_crust")
    cfg.update(precision="fp64", capacity=100000, sort_every=4, psi_break=[], f_break=[])
    o = oracle_mod.Oracle(cfg)
    ps = workloads.particles(cfg, seed=12)
    for s in range(2):
        o.set_particles(s, ps[s])
    for _ in range(3):
        o.step(4)
        d, _ = o.diagnostics()
        assert d.gauss_max < 1e-9 * d.rho_max, (d.gauss_max, d.rho_max)
    assert d.count[2] > 0 and d.injected > 0
