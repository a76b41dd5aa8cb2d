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
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="session")
def ihlib():
    """The built CUDA library (built on demand); a missing library fails."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_01656_gb300 import ih
    return ih


@pytest.fixture(scope="module")
def ctx(ihlib):
    import torch
    assert torch.cuda.is_available(), "a gpu-marked test needs a CUDA device"
    c = ihlib.ih_create(0)
    yield c
    ihlib.ih_destroy(c)
