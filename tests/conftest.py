import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size cases (minutes of host oracle time)")


@pytest.fixture(scope="session")
def lib():
    """The C-ABI library, built in-tree on first use (no GPU needed to load it)."""
    from paper_cs_0404008_gb300 import build as pkg_build
    pkg_build.build()
    from paper_cs_0404008_gb300 import gfpdot
    return gfpdot


@pytest.fixture(scope="session")
def ctx(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lib.Context(0)
    yield c
    c.close()
