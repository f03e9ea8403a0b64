import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 GPU and the CUDA library")
    config.addinivalue_line("markers", "slow: long-running (full-size) case")


def pytest_collection_modifyitems(config, items):
    """A gpu-marked test on a machine without a GPU is skipped, not failed."""
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def rt():
    """One runtime context on cuda:0 for the GPU tests (built on first use)."""
    import torch
    from paper_2106_03219_gb300 import build_lib
    from paper_2106_03219_gb300 import omprt as R
    build_lib.build()
    torch.cuda.init()
    r = R.Runtime(0)
    yield r
    torch.cuda.synchronize()
    r.close()
