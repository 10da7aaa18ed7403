"""The two ways of running the field update -- one fused, row-pipelined
pass over theta strips and row segments (field_pass 1) and J_perp before the
push plus four kernels after it (field_pass 2) -- give the same run, and the
automatic choice (field_pass 0) takes the fused pass only on grids large
enough to fill the GPU with it.

Whole steps with particles, injection and sorting, from the same seeded
state: after eight steps the fields agree to 1e-12 (FP64) or 1e-5 (FP32) in
relative L2, and the particles cell for cell (FP32: except within 1e-5 of a
face).  The grids have two theta strips and seven to nine row segments, so
halo columns and warm-up rows cross block boundaries every step."""
import numpy as np
import pytest

from helpers import FIELDS6, particle_mismatches, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,prec,tol", [("small_fine", "fp64", 1e-12), ("c1", "fp32", 1e-5)])
def test_fused_field_pass_equals_the_four_kernels(name, prec, tol):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_14512_gb300 import hff, workloads
    cfg = workloads.config(name)
    cfg.update(capacity=80000, precision=prec, sort_every=4, tile_r=8, tile_t=16)
    ps = workloads.particles(cfg, n_pairs=12000, seed=5)
    sims = []
    for fp in (1, 2):
        sim = hff.Sim(dict(cfg, field_pass=fp))
        assert sim.info().field_pass == fp
        for s in range(2):
            sim.load(s, ps[s])
        sim.step(8)
        assert sim.status() == 0
        sims.append(sim)
    a, b = sims
    for f in FIELDS6:
        assert rel_l2(b.get(f), a.get(f)) < tol, (f, rel_l2(b.get(f), a.get(f)))
    for s in range(2):
        pa, pb = a.particles(s), b.particles(s)
        assert np.count_nonzero(pa["cell"] >= 0) == np.count_nonzero(pb["cell"] >= 0)
        bad, ties, err = particle_mismatches(pb, pa, cfg["nt"])
        assert bad == 0, (s, bad, ties)
        assert err < (1e-5 if prec == "fp32" else 1e-11), err
    for sim in sims:
        sim.close()


def test_automatic_field_pass_follows_the_grid_size():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_14512_gb300 import hff, workloads
    for name, nr, nt, want in (("c1", 256, 128, hff.FIELDS_SPLIT), ("c1", 1024, 1024, hff.FIELDS_SPLIT),
                               ("c1", 2048, 2048, hff.FIELDS_FUSED)):
        cfg = dict(workloads.config(name), nr=nr, nt=nt, capacity=0, precision="fp32", sort_every=0)
        sim = hff.Sim(cfg)
        assert sim.info().field_pass == want, (nr, nt)
        sim.close()
