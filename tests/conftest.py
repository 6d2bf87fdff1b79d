import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# The oracle's OpenMP loops sleep rather than spin between regions, so a
# second process on the same cores does not stall them.
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line(
        "markers", "slow: long-running CPU physics check")


@pytest.fixture(scope="session")
def oracle_threads():
    """Oracle row loops use all host cores for the physics pins."""
    import oracle
    n = os.cpu_count() or 1
    oracle.set_threads(n)
    yield n
    oracle.set_threads(1)
