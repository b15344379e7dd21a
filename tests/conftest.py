import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def heget_lib():
    """Builds (if stale) and loads libheget.so."""
    from paper_0908_4403_gb300 import build, heget
    build.build()
    return heget


@pytest.fixture(scope="session")
def gpu(heget_lib):
    """A heget context on cuda:0 (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = heget_lib.heget_create(0)
    yield ctx
    torch.cuda.synchronize()
    heget_lib.heget_destroy(ctx)
