"""Edge cases of the C ABI on the GPU: an instance without particles,
capacity overflow latched by injection, a non-finite particle, the
radiation-reaction ramp scalar, grids that tiles do not divide, and FP64 /
FP32 instances of the same workload agreeing."""
import numpy as np
import pytest

from helpers import FIELDS6, rel_l2

pytestmark = pytest.mark.gpu
ST = dict(node=1, correct=2, push=4, faraday1=8, ampere=16, faraday2=32, inject=64, sort=128, all=255)


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


def test_no_particles_zero_capacity(env):
    hff, workloads, oracle = env
    cfg = workloads.config("small_hybrid")
    cfg.update(capacity=0, inject=False, sort_every=4)
    sim, ref = hff.Sim(cfg), oracle.Oracle(cfg)
    sim.load(0, {k: v[:0] for k, v in workloads.particles(cfg, n_pairs=1)[0].items()})
    sim.step(6)
    ref.step(6)
    # every field within the single-step tolerance after six steps (measured
    # at most 2.2e-7, E_ph, which starts at zero)
    for f in FIELDS6:
        assert rel_l2(sim.get(f), ref.get(f)) < 1e-5, f
    assert sim.status() == 0 and sim.info().count[0] == 0


def test_cell_outside_the_grid_is_rejected_on_load(env):
    """A caller's cell index at or past nr * nt is invalid: the load removes
    that particle, keeps the others in tile order and returns HFF_ERR_ARG;
    the instance then steps normally."""
    hff, workloads, _ = env
    for sort_every in (4, 0):
        cfg = workloads.config("small_hybrid")
        cfg.update(capacity=4000, inject=False, sort_every=sort_every)
        p = {k: v.copy() for k, v in workloads.particles(cfg, n_pairs=1500, seed=11)[0].items()}
        ncell = cfg["nr"] * cfg["nt"]
        p["cell"][[3, 500]] = [ncell, ncell + 12345]
        sim = hff.Sim(cfg)
        with pytest.raises(hff.HffError) as e:
            sim.load(0, p)
        assert e.value.code == hff.HFF_ERR_ARG
        got = sim.particles(0)
        assert int((got["cell"] >= 0).sum()) == 1498 and got["cell"].max() < ncell
        sim.step(3)
        assert sim.status() == 0
        sim.close()


def test_timed_step_is_the_production_step(env):
    """hff_step_timed replays the production step graph with two event-record
    nodes around the tiled push: the same result as hff_step (up to the order
    of the atomic sums) and positive push durations inside each step."""
    import torch
    hff, workloads, _ = env
    cfg = workloads.config("small_hybrid")
    cfg.update(capacity=40000, sort_every=4)
    ps = workloads.particles(cfg, n_pairs=5000, seed=8)
    a, b = hff.Sim(cfg), hff.Sim(cfg)
    for s in range(2):
        a.load(s, ps[s])
        b.load(s, ps[s])
    a.step(9)
    evb = [torch.cuda.Event(enable_timing=True) for _ in range(9)]
    eve = [torch.cuda.Event(enable_timing=True) for _ in range(9)]
    b.step_timed(evb, eve)
    torch.cuda.synchronize()
    for f in FIELDS6:
        assert rel_l2(b.get(f), a.get(f)) < 1e-5, f
    for s in range(2):
        ca, cb = a.particles(s)["cell"], b.particles(s)["cell"]
        assert len(ca) == len(cb) and np.mean(ca == cb) > 0.999
    ms = [evb[k].elapsed_time(eve[k]) for k in range(9)]
    assert all(m > 0 for m in ms)
    assert a.info().kernels_launched == b.info().kernels_launched
    a.close()
    b.close()


def test_capacity_overflow_is_latched(env):
    hff, workloads, _ = env
    cfg = workloads.config("small_pic")
    cfg.update(capacity=50, sort_every=0)   # the first injection needs far more
    sim = hff.Sim(cfg)
    sim.step(1)
    assert sim.status() == hff.HFF_ERR_CAPACITY
    assert sim.info().count[0] == 50
    assert sim.status() == 0                 # read-and-clear


def test_nonfinite_particle_removed_and_flagged(env):
    hff, workloads, _ = env
    cfg = workloads.config("small_pic")
    cfg.update(capacity=100, inject=False, sort_every=0)
    sim = hff.Sim(cfg)
    p = workloads.particles(cfg, n_pairs=10, seed=3)[0]
    p = {k: v.copy() for k, v in p.items()}
    p["ur"] = p["ur"].astype(np.float64)
    p["ur"][4] = np.nan
    sim.load(0, p)
    sim.step_stages(1, ST["node"] | ST["push"])
    g = sim.particles(0)
    assert g["cell"][4] == -1 and np.all(g["cell"][np.arange(10) != 4] >= 0)
    assert sim.status() == hff.HFF_ERR_NONFINITE
    d, _ = sim.diagnostics()
    assert d.nonfinite == 1.0


def test_rr_scale_zero_equals_no_radiation(env):
    hff, workloads, _ = env
    cfg = workloads.config("small_rr")
    cfg.update(capacity=20000, inject=False, sort_every=0)
    ps = workloads.particles(cfg, n_pairs=4000, seed=9)
    a = hff.Sim(cfg)
    b = hff.Sim(dict(cfg, gamma_rad=0.0))
    a.set_rr_scale(0.0)
    for s in range(2):
        a.load(s, ps[s])
        b.load(s, ps[s])
    a.step_stages(1, ST["node"] | ST["push"])
    b.step_stages(1, ST["node"] | ST["push"])
    for s in range(2):
        pa, pb = a.particles(s), b.particles(s)
        for k in ("cell", "xo", "yo", "ur", "ut", "up"):
            assert np.array_equal(pa[k], pb[k]), k
    a.set_rr_scale(1.0)
    a.step_stages(1, ST["node"] | ST["push"])
    b.step_stages(1, ST["node"] | ST["push"])
    assert not np.array_equal(a.particles(0)["ur"], b.particles(0)["ur"])


@pytest.mark.parametrize("tiles", [(5, 7), (16, 32), (40, 56)])
def test_ragged_tiles_same_result(env, tiles):
    """The tile shape changes only the particle order within the sorted
    array; the fields after whole steps agree with the oracle for tile
    shapes that do not divide the grid."""
    hff, workloads, oracle = env
    cfg = workloads.config("small_hybrid")
    cfg.update(capacity=40000, sort_every=3, tile_r=tiles[0], tile_t=tiles[1])
    ps = workloads.particles(cfg, n_pairs=6000, seed=13)
    sim, ref = hff.Sim(cfg), oracle.Oracle(cfg)
    for s in range(2):
        sim.load(s, ps[s])
        ref.set_particles(s, ps[s])
    ref.sort_now()
    sim.step(7)
    ref.step(7)
    for f in FIELDS6:
        assert rel_l2(sim.get(f), ref.get(f)) < 1e-5, f
    for s in range(2):
        assert np.array_equal(sim.particles(s)["cell"].shape, ref.particles(s)["cell"].shape)


def test_fp32_and_fp64_instances_agree(env):
    """The FP32 production path against the FP64 instantiation of the same
    kernels over ten steps of the hybrid workload (diagnostics within 1e-4)."""
    hff, workloads, _ = env
    cfg = workloads.config("small_hybrid")
    cfg.update(capacity=60000, sort_every=4)
    ps = workloads.particles(cfg, n_pairs=8000, seed=17)
    s32, s64 = hff.Sim(cfg), hff.Sim(dict(cfg, precision="fp64"))
    for s in range(2):
        s32.load(s, ps[s])
        s64.load(s, ps[s])
    s32.step(10)
    s64.step(10)
    d32, l32 = s32.diagnostics()
    d64, l64 = s64.diagnostics()
    assert rel_l2(l32, l64) < 1e-5
    assert abs(d32.psi_open - d64.psi_open) < 1e-5 * abs(d64.psi_open)
    for f in FIELDS6:
        assert rel_l2(s32.get(f), s64.get(f)) < 1e-5, f


def test_deferred_gather_same_state(env):
    """A sort leaves its payload gather to the next push; reading the
    particles in between performs the gather eagerly instead.  Both routes
    give the same state (FP64: up to the rounding of the atomic deposit
    order)."""
    hff, workloads, _ = env
    cfg = workloads.config("small_pic")
    cfg.update(capacity=40000, sort_every=4, precision="fp64")
    ps = workloads.particles(cfg, n_pairs=6000, seed=41)
    runs = []
    for mode in ("straight", "read", "diag"):
        sim = hff.Sim(cfg)
        for s in range(2):
            sim.load(s, ps[s])
        sim.step(4)                       # ends with a sort: gather pending
        if mode == "read":
            sim.particles(1)
        elif mode == "diag":
            sim.diagnostics()
        sim.step(5)
        runs.append(({s: sim.particles(s) for s in range(2)}, {f: sim.get(f) for f in ("E_r", "E_ph", "B_th")}))
        assert sim.status() == 0
        sim.close()
    ref_p, ref_f = runs[0]
    for parts, fields in runs[1:]:
        for s in range(2):
            assert np.array_equal(parts[s]["cell"], ref_p[s]["cell"])
            for k in ("xo", "yo", "ur", "ut", "up", "w"):
                np.testing.assert_allclose(parts[s][k], ref_p[s][k], rtol=1e-12, atol=1e-14)
        for f in fields:
            np.testing.assert_allclose(fields[f], ref_f[f], rtol=1e-11, atol=1e-14)


def test_clamp_counter_matches_oracle(env):
    """The running count of Eq. 26 activations equals the oracle's in FP64
    over ten hybrid steps (same decisions at every node)."""
    hff, workloads, oracle = env
    cfg = workloads.config("small_hybrid")
    cfg.update(capacity=40000, sort_every=4, precision="fp64")
    ps = workloads.particles(cfg, n_pairs=4000, seed=43)
    sim, ref = hff.Sim(cfg), oracle.Oracle(cfg)
    for s in range(2):
        sim.load(s, ps[s])
        ref.set_particles(s, ps[s])
    ref.sort_now()
    sim.step(10)
    ref.step(10)
    g, o = sim.diagnostics()[0], ref.diagnostics()[0]
    assert o.clamps > 0
    assert g.clamps == o.clamps, (g.clamps, o.clamps)
    assert g.nonfinite_fields == 0


def test_nonfinite_field_is_detected_and_latched(env):
    hff, workloads, _ = env
    cfg = workloads.config("small_pic")
    cfg.update(capacity=100, sort_every=0)
    sim = hff.Sim(cfg)
    er = sim.get("E_r")
    er[5, 7] = np.nan
    sim.set("E_r", er)
    d, _ = sim.diagnostics()
    assert d.nonfinite_fields >= 1
    assert sim.status() == hff.HFF_ERR_NONFINITE
    assert "field" in hff.hff_last_error()
    assert sim.status() == 0
