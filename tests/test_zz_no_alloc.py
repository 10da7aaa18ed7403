"""The allocation-free tile ordering (hff_tile_order_noalloc) against the
ordering that hff_load_particles applies, through the C ABI.

Some callers may not allocate device memory at all (an application that
owns every allocation, or runs under a budget that forbids ad-hoc
cudaMalloc); this entry point keeps its scratch in a fixed array inside the
library.  The test runs two calls in a row on different inputs, so that a
call that depended on what the previous one left in the shared array would
fail, and checks the size limit.  It lives in its own file, collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_14512_gb300 import hff, workloads
    return torch, hff, workloads


def test_noalloc_order_matches_load_sort(env):
    torch, hff, workloads = env
    cfg = workloads.config("small_hybrid")
    cfg.update(capacity=40000, sort_every=4, inject=False, tile_r=8, tile_t=16)
    ps = workloads.particles(cfg, n_pairs=12000, seed=77)
    stream = torch.cuda.current_stream()
    for call, (species, drop) in enumerate([(0, 3), (1, 7)]):
        p = {k: v.copy() for k, v in ps[species].items()}
        p["cell"][::drop] = -1
        if call == 1:  # a different arrangement of the same particles
            perm = np.random.default_rng(5).permutation(len(p["cell"]))
            p = {k: v[perm].copy() for k, v in p.items()}
        sim = hff.Sim(cfg)
        sim.load(0, p)                         # existing entry point: sorts on load
        ref = sim.particles(0)
        cell = torch.from_numpy(p["cell"]).cuda()
        order = torch.empty(len(p["cell"]), dtype=torch.int32, device="cuda")
        live = hff.hff_tile_order_noalloc(cell.data_ptr(), cell.numel(), cfg["nr"], cfg["nt"],
                                          cfg["tile_r"], cfg["tile_t"], order.data_ptr(), stream.cuda_stream)
        o = order.cpu().numpy()[:live]
        assert live == len(ref["cell"]) == int(np.sum(p["cell"] >= 0))
        assert np.array_equal(p["cell"][o], ref["cell"])
        assert np.array_equal(p["xo"][o], ref["xo"]) and np.array_equal(p["w"][o], ref["w"])
        sim.close()


def test_noalloc_rejects_oversized_input(env):
    torch, hff, _ = env
    n = hff.NOALLOC_MAX_PARTICLES + 1
    cell = torch.zeros(n, dtype=torch.int32, device="cuda")
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(hff.HffError) as e:
        hff.hff_tile_order_noalloc(cell.data_ptr(), n, 64, 64, 8, 8, order.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert e.value.code == hff.HFF_ERR_CAPACITY


def test_noalloc_rejects_a_cell_outside_the_grid(env):
    """A cell index at or past nr * nt orders as removed and the call reports
    HFF_ERR_ARG; a valid call right after it still matches the load order."""
    torch, hff, _ = env
    nr, nt = 64, 48
    cell = torch.arange(0, 3000, dtype=torch.int32, device="cuda")
    cell[17] = nr * nt + 5
    order = torch.empty(3000, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    with pytest.raises(hff.HffError) as e:
        hff.hff_tile_order_noalloc(cell.data_ptr(), 3000, nr, nt, 8, 8, order.data_ptr(), st)
    assert e.value.code == hff.HFF_ERR_ARG
    assert int(order[2999].item()) == 17           # ordered last, with the removed ones
    cell[17] = 17
    live = hff.hff_tile_order_noalloc(cell.data_ptr(), 3000, nr, nt, 8, 8, order.data_ptr(), st)
    assert live == 3000
    c = cell.cpu().numpy()
    key = (c // nt // 8) * ((nt + 7) // 8) + (c % nt) // 8
    assert np.array_equal(order.cpu().numpy(), np.argsort(key, kind="stable"))
