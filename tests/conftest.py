import os
import sys

# one hardware work queue per concurrent stream, before CUDA initialises
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")

import pytest


@pytest.fixture(scope="session")
def sgctx():
    """One library context on cuda:0 (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_18155_gb300 import build
    build.build()
    from paper_2406_18155_gb300.api import Context
    c = Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()
