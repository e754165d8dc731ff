"""Shared test setup: markers, import path, oracle build."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def orc():
    """The CPU oracle, built once per session."""
    import oracle
    oracle.build()
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def libdose():
    """The CUDA engine's C-ABI library, built in-tree (nvcc cross-compiles
    without a GPU) and loaded through the thin binding."""
    from paper_1809_03927_gb300 import build
    build.build()
    from paper_1809_03927_gb300 import dose
    return dose


@pytest.fixture(scope="session")
def gpu(libdose):
    """Skip unless a CUDA device is usable; returns the binding."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return libdose
