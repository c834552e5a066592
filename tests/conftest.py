import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check (tens of seconds)")


@pytest.fixture(scope="session")
def lblib():
    """Build (if stale) and load libthermal_lbm.so."""
    from paper_1111_0905_gb300 import build, lb
    build.build()
    return lb.load_library()


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for tests marked gpu")
    return torch
