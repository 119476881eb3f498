import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def banded_4m_host():
    """The full-size banded workload (n = 2^22, m = 8, 16 successors in a +-4096 band)."""
    import synth
    return synth.banded_4m()


@pytest.fixture(scope="session")
def banded_4m_gpu(banded_4m_host):
    from paper_2502_14474_gb300 import MDP
    h = MDP.from_csr(banded_4m_host)
    yield banded_4m_host, h
    h.close()
