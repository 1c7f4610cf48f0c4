import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


@pytest.fixture(scope="session", autouse=True)
def built_libraries():
    """Build the CUDA library and the oracle if missing or stale (no-ops when
    they are up to date), so that every test runs against current binaries."""
    from paper_1405_2912_b300 import build
    build.build()
    import oracle
    oracle.build()


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle
