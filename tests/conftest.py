import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: a CPU test that takes more than a few seconds")


def pytest_collection_modifyitems(config, items):
    # GPU tests skip cleanly on a machine without a GPU only when explicitly
    # deselected; when selected (-m gpu) they must run and fail loudly.
    pass


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle
