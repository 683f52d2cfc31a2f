import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


# GPU modules that run after all the others, in this order: rejected inputs,
# the counting sweep (sixty extractions up to 5e6 edges), the polyhedral
# domains, then the counting sweep at D = 5 and 6
# and last of all the allocation-free entry point, so that a run that stops at
# its first failure has run every other test before it
_LAST = {"test_gpu_invalid_inputs.py": 1, "test_gpu_counting_sweep.py": 2, "test_gpu_domains.py": 3,
         "test_gpu_counting_sweep_high_dims.py": 4, "test_zz_no_alloc.py": 5}


def pytest_collection_modifyitems(config, items):
    # the sort is stable, so every other order is kept
    items.sort(key=lambda it: _LAST.get(os.path.basename(str(it.fspath)), 0))
