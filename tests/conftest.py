import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libmclbm.so")
    config.addinivalue_line("markers", "slow: long-running oracle pin")


@pytest.fixture(scope="session")
def gpu_lib():
    """Build (if stale) and load the CUDA library; skip nothing silently."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu test collected on a machine without CUDA")
    from paper_1601_01237_gb300 import build
    build.build()
    from paper_1601_01237_gb300 import _native
    return _native.lib()
