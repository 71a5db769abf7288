import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libgraphstep")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle():
    import oracle as _oracle

    _oracle.build()
    return _oracle


@pytest.fixture(scope="session")
def fdtd_config2_ref(oracle):
    """FP64 oracle of the 128^3 driven cavity after 5000 steps (computed once)."""
    N, n, src = 128, 5000, (64, 64, 64)
    return oracle.fdtd_run(oracle.fdtd_zero_fields(N), N, n, src=src)
