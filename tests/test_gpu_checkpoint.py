"""Checkpoint / resume and the density, energy and spectrum diagnostics
through the C ABI.

Resume: a run saved at step 6 and continued for 7 steps must equal a fresh
instance restored from the blob and stepped 7 times (FP64: to the rounding
of the atomic deposit order; FP32: within 1e-5), with injection and pair
creation on, across sorts.  Maps and spectra: against the oracle on the
same particles."""
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


def pairs_cfg(workloads, precision):
    cfg = workloads.config("small_pairs")
    cfg.update(precision=precision, sort_every=4, capacity=80000, gamma_rad=0.0)
    return cfg


def state(sim):
    return ({s: sim.particles(s) for s in range(2)}, {f: sim.get(f) for f in FIELDS6}, sim.diagnostics()[0])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_resume_equals_continuing(env, precision, tol):
    hff, workloads, _ = env
    cfg = pairs_cfg(workloads, precision)
    ps = workloads.particles(cfg, seed=31)
    a = hff.Sim(cfg)
    for s in range(2):
        a.load(s, ps[s])
    a.step(6)                      # 6 is not a multiple of 4: the tail is unsorted
    blob = a.checkpoint()
    a.step(7)
    b = hff.Sim(dict(cfg, capacity=90000))   # capacity may differ
    b.restore(blob)
    assert b.info().step == 6
    b.step(7)
    assert b.info().step == a.info().step == 13
    pa, fa, da = state(a)
    pb, fb, db = state(b)
    for s in range(2):
        if precision == "fp64":
            assert np.array_equal(pa[s]["cell"], pb[s]["cell"]), s
        else:   # FP32 deposit-order rounding may move a particle across a face it touches
            bad, ties, err = particle_mismatches(pb[s], pa[s], cfg["nt"])
            assert bad == 0 and ties <= 2 and err < 1e-5, (s, bad, ties, err)
        same = pa[s]["cell"] == pb[s]["cell"]
        for k in ("xo", "yo", "ur", "ut", "up", "w"):
            assert rel_l2(pb[s][k][same], pa[s][k][same]) < tol, (s, k)
    for f in FIELDS6:
        assert rel_l2(fb[f], fa[f]) < tol, f
    for k in ("injected", "created", "killed"):
        assert abs(getattr(db, k) - getattr(da, k)) <= tol * max(1.0, abs(getattr(da, k))), k
    assert da.created > 0 and da.injected > 0
    assert a.status() == 0 and b.status() == 0
    a.close()
    b.close()


def test_checkpoint_file_round_trip_and_rejections(env, tmp_path):
    hff, workloads, _ = env
    cfg = pairs_cfg(workloads, "fp32")
    ps = workloads.particles(cfg, seed=32)
    a = hff.Sim(cfg)
    for s in range(2):
        a.load(s, ps[s])
    a.step(3)
    path = str(tmp_path / "run.ckpt")
    a.save(path)
    b = hff.Sim(cfg)
    b.resume(path)
    for s in range(2):
        x, y = a.particles(s), b.particles(s)
        for k in x:
            assert np.array_equal(x[k], y[k]), (s, k)
    for f in FIELDS6:
        assert np.array_equal(a.get(f), b.get(f)), f
    blob = a.checkpoint()
    with pytest.raises(hff.HffError, match="different configuration"):
        hff.Sim(dict(cfg, r_lc=cfg["r_lc"] * 1.01)).restore(blob)
    with pytest.raises(hff.HffError, match="truncated"):
        b.restore(blob[:-100])
    with pytest.raises(hff.HffError, match="not a checkpoint"):
        b.restore(np.zeros(4096, np.uint8))
    small = hff.Sim(dict(cfg, capacity=100))
    with pytest.raises(hff.HffError) as e:
        small.restore(blob)
    assert e.value.code == hff.HFF_ERR_CAPACITY


def test_ensemble_member_resumes_alone(env):
    hff, workloads, _ = env
    cfgs = workloads.ensemble("small_c5")
    for c in cfgs:
        c.update(sort_every=4, capacity=30000, precision="fp64")
    ens = hff.Ensemble(cfgs)
    for k, c in enumerate(cfgs):
        ps = workloads.particles(c, seed=c["seed"] + 7)
        for s in range(2):
            ens[k].load(s, ps[s])
    ens.step(5)
    blob = ens[2].checkpoint()
    ens.step(3)
    lone = hff.Sim(cfgs[2])
    lone.restore(blob)
    lone.step(3)
    for f in FIELDS6:
        assert rel_l2(lone.get(f), ens[2].get(f)) < 1e-12, f
    for s in range(2):
        assert np.array_equal(lone.particles(s)["cell"], ens[2].particles(s)["cell"])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_maps_and_spectrum_match_oracle(env, precision):
    hff, workloads, oracle = env
    cfg = workloads.config("small_rr")
    cfg.update(precision=precision, capacity=40000, sort_every=4)
    ps = workloads.particles(cfg, seed=33)
    sim, ref = hff.Sim(cfg), oracle.Oracle(cfg)
    for s in range(2):
        sim.load(s, ps[s])
        ref.set_particles(s, ps[s])
    ref.sort_now()
    for s in range(2):
        gd, ge = sim.species_maps(s)
        od, oe = ref.species_maps(s)
        assert rel_l2(gd, od) < 1e-12 and rel_l2(ge, oe) < 1e-10, s
        gs, os_ = sim.spectrum(s, 48, 0.0, 6.0), ref.spectrum(s, 48, 0.0, 6.0)
        assert abs(gs.sum() - os_.sum()) < 1e-12 * os_.sum()
        assert rel_l2(gs, os_) < 1e-12, s
    if precision == "fp64":   # after steps, the FP64 instance still agrees
        sim.step(5)
        ref.step(5)
        for s in range(2):
            gd, ge = sim.species_maps(s)
            od, oe = ref.species_maps(s)
            assert rel_l2(gd, od) < 1e-9 and rel_l2(ge, oe) < 1e-9, s
