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


@pytest.hookimpl(trylast=True)   # after -m / -k have deselected
def pytest_collection_modifyitems(session, config, items):
    # the full-size oracle runs take minutes of host time: start them as soon
    # as such tests are selected, so that they overlap the other GPU tests
    if any(item.get_closest_marker("fullsize") for item in items):
        import torch
        if torch.cuda.is_available():
            from tests import fullsize_oracle
            fullsize_oracle.start("lwa")
            fullsize_oracle.start("large_n")
