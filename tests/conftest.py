import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# collected after every other test, full-size cases included
LAST_FILE = "test_zz_no_alloc.py"


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libdgcns")
    config.addinivalue_line("markers", "slow: takes more than ~20 s on the CPU")
    config.addinivalue_line("markers", "full_size: runs the benchmark workload at full size (run after the small cases)")


def pytest_collection_modifyitems(config, items):
    """Full-size cases run after every small case, and the file LAST_FILE after everything (stable order
    otherwise)."""
    items.sort(key=lambda it: (os.path.basename(str(it.fspath)) == LAST_FILE,
                               it.get_closest_marker("full_size") is not None))
