"""Ensembles: independent instances stepped together by one graph launch per
step.  Each member must reproduce the FP64 oracle exactly as a lone instance
does, and an FP64 ensemble must give the results of the same instances run
one by one (the graph branches share nothing)."""
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


def small(workloads, **kw):
    cfgs = workloads.ensemble("small_c5")
    for c in cfgs:
        c.update(sort_every=4, capacity=30000, **kw)
    return cfgs


def inputs(workloads, cfgs):
    return [workloads.particles(c, seed=c["seed"] + 100) for c in cfgs]


def test_ensemble_members_match_oracle(env):
    hff, workloads, oracle = env
    cfgs = small(workloads)
    ps = inputs(workloads, cfgs)
    ens = hff.Ensemble(cfgs)
    refs = []
    for k, c in enumerate(cfgs):
        ref = oracle.Oracle(c)
        for s in range(2):
            ens[k].load(s, ps[k][s])
            ref.set_particles(s, ps[k][s])
        ref.sort_now()
        refs.append(ref)
    ens.step(10)
    info = ens.info()
    assert info.n_inst == len(cfgs) and info.step == 10
    for k, ref in enumerate(refs):
        ref.step(10)
        for s in range(2):
            g, o = ens[k].particles(s), ref.particles(s)
            bad, ties, err = particle_mismatches(g, o, cfgs[k]["nt"])
            assert bad == 0 and ties <= max(2, len(o["cell"]) // 2000), (k, s, bad, ties)
            assert err < 1e-5, (k, err)
        # FP32 over ten steps: the single-step tolerance, as for a lone instance
        errs = {f: rel_l2(ens[k].get(f), ref.get(f)) for f in FIELDS6}
        assert max(errs.values()) < 1e-5, (k, errs)
    assert ens.status() == 0
    assert info.count[0] == sum(int(ens[k].particle_views(0)["cell"].numel()) for k in range(len(cfgs)))
    ens.close()


def test_fp64_ensemble_equals_lone_instances(env):
    """Same inputs, FP64: ensemble members and lone instances agree to the
    rounding of the deposit's atomic order; only some members get particles,
    so the members start on different buffer parities."""
    hff, workloads, _ = env
    cfgs = small(workloads, precision="fp64")
    ps = inputs(workloads, cfgs)
    ens = hff.Ensemble(cfgs)
    lone = [hff.Sim(c) for c in cfgs]
    for k in range(len(cfgs)):
        species = (0, 1) if k % 2 == 0 else (1,)
        for s in species:
            ens[k].load(s, ps[k][s])
            lone[k].load(s, ps[k][s])
    ens.step(9)
    for sim in lone:
        sim.step(9)
    for k, sim in enumerate(lone):
        for f in FIELDS6:
            assert rel_l2(ens[k].get(f), sim.get(f)) < 1e-12, (k, f)
        for s in range(2):
            a, b = ens[k].particles(s), sim.particles(s)
            assert np.array_equal(a["cell"], b["cell"]), (k, s)
            for q in ("xo", "yo", "ur", "ut", "up", "w"):
                np.testing.assert_allclose(a[q], b[q], rtol=1e-12, atol=1e-12)
        sim.close()
    ens.close()


def test_ensemble_status_names_the_instance(env):
    """A capacity overflow in one member is latched and reported with the
    member's index; reading the status clears every member."""
    hff, workloads, _ = env
    cfgs = small(workloads)
    cfgs[2]["capacity"] = 4             # a handful of polar-cap cells inject more than that
    ens = hff.Ensemble(cfgs)
    ens.step(2)
    assert ens.status() == hff.HFF_ERR_CAPACITY
    assert "instance 2" in hff.hff_last_error()
    assert ens.status() == 0
    ens.close()


def test_ensemble_rejects_mixed_precision(env):
    hff, workloads, _ = env
    cfgs = small(workloads)
    cfgs[1]["precision"] = "fp64"
    with pytest.raises(hff.HffError, match="share precision"):
        hff.Ensemble(cfgs)


def test_c5_ensemble_full_size(env):
    """The 32-instance workload at full size: one graph launch per step; the
    four members with the fewest particles checked against the oracle after a
    whole step, every member clean after a further 16 steps (two sorts)."""
    hff, workloads, oracle = env
    cfgs = workloads.ensemble("c5")
    ens = hff.Ensemble(cfgs)
    ps = [workloads.particles(c) for c in cfgs]
    for k in range(len(cfgs)):
        for s in range(2):
            ens[k].load(s, ps[k][s])
    picks = sorted(range(len(cfgs)), key=lambda k: cfgs[k]["n_pairs"])[:4]
    refs = {}
    for k in picks:
        ref = oracle.Oracle(cfgs[k])
        for s in range(2):
            ref.set_particles(s, ps[k][s])
        ref.sort_now()
        refs[k] = ref
    ens.step(1)
    for k, ref in refs.items():
        ref.step(1)
        for s in range(2):
            g, o = ens[k].particles(s), ref.particles(s)
            bad, ties, err = particle_mismatches(g, o, cfgs[k]["nt"])
            assert bad == 0 and ties <= max(2, len(o["cell"]) // 2000), (k, s, bad, ties)
            assert err < 1e-5, (k, err)
        # every field, E_ph (which starts at zero) included, within 1e-5
        errs = {f: rel_l2(ens[k].get(f), ref.get(f)) for f in FIELDS6}
        for f, e in errs.items():
            assert e < 1e-5, (k, f, e)
    ens.step(16)
    assert ens.status() == 0
    info = ens.info()
    assert info.step == 17 and info.n_inst == 32
    for k in range(len(cfgs)):
        d, _ = ens[k].diagnostics()
        assert d.nonfinite == 0
        assert d.count[0] > 0.5 * cfgs[k]["n_pairs"]
    ens.close()
