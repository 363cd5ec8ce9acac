import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: oracle work of more than a few seconds")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="session")
def ctx():
    """A library context on cuda:0 (GPU tests only)."""
    import torch
    import paper_2402_09356_gb300 as tlr
    from paper_2402_09356_gb300 import build as tlr_build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tlr_build.build()
    torch.cuda.init()
    c = tlr.Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()
