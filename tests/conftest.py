import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_modifyitems(config, items):
    # keep the file named test_zz_* last, whatever the ordering plugins do
    items.sort(key=lambda it: os.path.basename(str(it.fspath)).startswith("test_zz_"))
