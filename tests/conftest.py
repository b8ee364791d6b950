import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (run with -m gpu on a GB300)")
    config.addinivalue_line("markers", "slow: large inputs (full benchmark sizes)")


@pytest.fixture(scope="session")
def rmat12():
    import gen
    return gen.rmat(12, 16)
