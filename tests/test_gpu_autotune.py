"""The launch-shape autotuner times every candidate it is given and returns
the fastest one that fits; oversized tiles are reported, not fatal."""
import pytest

pytestmark = pytest.mark.gpu


def test_autotune_small_sample():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_14512_gb300 import autotune
    res = autotune.tune("c3", grid=256, tiles=[(8, 16), (16, 32), (64, 128)], cadences=[2, 8],
                        steps=8, warmup=2)
    table = res["table"]
    assert len(table) == 6
    timed = [t for t in table if t["ms_per_step"] is not None]
    assert len(timed) >= 4
    assert all(t["ms_per_step"] > 0 for t in timed)
    assert res["best"]["ms_per_step"] == min(t["ms_per_step"] for t in timed)
    # 64 x 128 tiles with their halo exceed the shared memory of one block
    assert any(t["tile_r"] == 64 and t["ms_per_step"] is None for t in table)


def test_init_path_measures_caches_and_builds():
    """A configuration with tile_r = tile_t = 0 and sort_every = -1 gets the
    fastest measured shape on the caller's particles; a second request is
    served from the cache; Sim(cfg, particles=...) builds with that shape."""
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_14512_gb300 import autotune, hff, workloads
    cfg = workloads.config("small_hybrid")
    cfg.update(capacity=60000, tile_r=0, tile_t=0, sort_every=autotune.AUTO, nr=120)
    ps = workloads.particles(cfg, n_pairs=20000, seed=3)
    if os.path.exists(autotune.CACHE):
        os.remove(autotune.CACHE)
    tiles, cads = [(8, 16), (16, 16), (16, 32)], [4, 8]
    got = autotune.resolve(cfg, ps, tiles=tiles, cadences=cads, steps=8, warmup=2)
    info = got["autotune"]
    assert info["source"] == "measured" and len(info["table"]) == 6
    timed = [t for t in info["table"] if t["ms_per_step"] is not None]
    best = min(timed, key=lambda t: t["ms_per_step"])
    assert (got["tile_r"], got["tile_t"], got["sort_every"]) == (best["tile_r"], best["tile_t"], best["sort_every"])
    again = autotune.resolve(cfg, ps, tiles=tiles, cadences=cads)
    assert again["autotune"]["source"] == "cache"
    assert (again["tile_r"], again["tile_t"], again["sort_every"]) == (got["tile_r"], got["tile_t"], got["sort_every"])
    sim = hff.Sim(cfg, particles=ps)
    assert (sim.cfg["tile_r"], sim.cfg["tile_t"], sim.cfg["sort_every"]) == (got["tile_r"], got["tile_t"], got["sort_every"])
    info_c = sim.info()
    assert (info_c.tile_r, info_c.tile_t, info_c.sort_every) == (got["tile_r"], got["tile_t"], got["sort_every"])
    sim.close()
    # without particles and without a cached entry: the documented fallback
    os.remove(autotune.CACHE)
    fb = autotune.resolve(cfg)
    assert (fb["tile_r"], fb["tile_t"], fb["sort_every"]) == autotune.DEFAULT_SHAPE
