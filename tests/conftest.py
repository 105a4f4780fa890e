import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def ng():
    """The CUDA library binding (built in-tree first); GPU tests only."""
    import torch
    from paper_2101_10994_gb300 import build, nglod
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return nglod
