"""The package entry point's smoke check on the GPU: one small FP64 run of the fused step
(16 x 10 x 12 boiling cell, 5 steps) against the oracle, fields within 1e-12 and Nu within 1e-9."""
import pytest


@pytest.mark.gpu
def test_smoke_entry_point(cuda, lblib):
    import __graft_entry__ as entry
    entry.smoke()
