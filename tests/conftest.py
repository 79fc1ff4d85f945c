import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for _p in (ROOT, os.path.join(ROOT, "tests")):
    if _p not in sys.path:
        sys.path.insert(0, _p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libhelrm.so")
    config.addinivalue_line("markers", "slow: long CPU-only oracle runs")


@pytest.fixture(scope="session")
def small_params():
    """N = 2^10 with the full chain's prime shape (60-bit base, 40-bit levels,
    three 60-bit special primes, alpha = 3)."""
    from oracle import ckks
    return ckks.Params(10, [60] + [40] * 5, 3, 60, 3, 40.0)


@pytest.fixture(scope="session")
def small_keys(small_params):
    from oracle import ckks
    return ckks.keygen(small_params, 1234, rot_steps=[1, 2, 3, 5, -1, -7, 100])
