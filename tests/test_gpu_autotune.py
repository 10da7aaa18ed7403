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
