import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: larger cases (a minute or two at most)")


def pytest_collection_modifyitems(config, items):
    # keep whatever order pytest chose, but run files whose name sorts last
    # (test_zz_*) after every other file
    items.sort(key=lambda it: os.path.basename(str(it.fspath)).startswith("test_zz_"))
