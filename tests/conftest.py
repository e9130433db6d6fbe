import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libwl.so")
    config.addinivalue_line("markers", "slow: long-running oracle case")


import pytest


@pytest.fixture(scope="session", autouse=True)
def _build_native():
    """Build libwl.so and the oracle library in-tree (incremental; no GPU needed)."""
    from paper_2304_08159_gb300 import build
    import oracle

    build.build_all()
    oracle.build()
