import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU-only test")


def has_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library; a GPU test fails (never skips to a fallback) if it cannot load."""
    if not has_gpu():
        pytest.fail("gpu test selected but no CUDA device is visible")
    import paper_2408_01470_b300 as lib
    lib.load()
    return lib
