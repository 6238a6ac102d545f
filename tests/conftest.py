"""Shared fixtures.  Tests marked ``gpu`` need a GB300 and the CUDA library;
everything else runs on the CPU (oracle pins, host logic, ABI exports)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def gmq_lib():
    """The built C-ABI library (ctypes), without touching the GPU."""
    from paper_2511_01573_gb300 import gmq
    return gmq


@pytest.fixture(scope="session")
def gpu_ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_01573_gb300 import gmq
    ctx = gmq.Context(device=0)
    yield ctx
    ctx.close()
