import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def kbc():
    """The CUDA library binding; GPU tests fail loudly if it cannot be loaded."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_1507_02518_gb300 as pkg
    pkg.lb.load()  # raises if libkbc.so is missing or broken
    return pkg
