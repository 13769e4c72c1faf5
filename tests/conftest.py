import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built tweedmg library")
    config.addinivalue_line("markers", "slow: long CPU test (full tables)")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def mg():
    """The CUDA library through its Python binding (built in-tree on first use)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2110_08389_gb300 import build, mg as mgmod
    build.build()
    mgmod.load()
    return mgmod
