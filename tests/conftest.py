import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: test that takes more than a few seconds")
    # the library is compiled in-tree (nvcc cross-compiles without a GPU); test
    # modules that import the binding at collection need it to exist
    from paper_1312_1476_gb300 import _build
    _build.build()


def pytest_collection_modifyitems(config, items):
    # Nothing to skip automatically: -m gpu / -m "not gpu" selects.
    return None
