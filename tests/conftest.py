import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libfcgno.so")


@pytest.fixture(scope="session")
def lib():
    """The CUDA binding; GPU tests fail loudly if the library is missing."""
    from paper_2402_05598_gb300 import fcgno
    return fcgno


@pytest.fixture(scope="session")
def dev():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    return torch.device("cuda:0")
