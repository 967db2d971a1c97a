import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a) and the built libmsz.so")
    config.addinivalue_line("markers", "slow: large case; still part of the default run")


def pytest_collection_modifyitems(config, items):
    # a gpu test without a GPU is a configuration error, not a skip, when -m gpu is asked for
    pass


@pytest.fixture(scope="session")
def msz():
    """The product's Python binding; loading it fails loudly without libmsz.so."""
    import paper_2601_01787_gb300 as m
    return m
