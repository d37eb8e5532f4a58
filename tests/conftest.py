import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libfpm")
    config.addinivalue_line("markers", "slow: long-running CPU oracle comparisons")


@pytest.fixture(scope="session")
def libfpm():
    """Build (if stale) and load libfpm.so."""
    from paper_2010_11847_gb300 import build, binding
    build.build()
    return binding.lib()


@pytest.fixture(scope="session")
def cuda(libfpm):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    torch.cuda.init()
    return torch.device("cuda", 0)
