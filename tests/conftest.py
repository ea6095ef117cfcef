import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: large CPU-side case")


def pytest_collection_modifyitems(config, items):
    # run every gpu test after the CPU ones so a GPU failure does not hide them
    items.sort(key=lambda it: 1 if it.get_closest_marker("gpu") else 0)
