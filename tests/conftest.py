import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA device (B300, sm_103a) and the built library")
    config.addinivalue_line(
        "markers", "fullsize: full-size workloads checked over every baseline (minutes of oracle time)")


@pytest.fixture(scope="session")
def gpu_available():
    import torch
    return torch.cuda.is_available()
