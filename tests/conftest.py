import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def nb():
    """The CUDA library binding; a GPU test fails (not skips) when the GPU is
    present but the library cannot be loaded."""
    if not _cuda_ok():
        pytest.skip("no CUDA device")
    import paper_2411_18889_gb300 as nbody
    nbody.load()  # raises if the shared library is missing
    return nbody
