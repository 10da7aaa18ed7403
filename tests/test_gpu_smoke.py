"""The round-trip check __graft_entry__.smoke() runs on a fresh GPU: one small
hybrid instance through the C ABI against the oracle for four steps."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    __graft_entry__.smoke()
