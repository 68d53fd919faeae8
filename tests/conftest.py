import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes tens of seconds")


def pytest_collection_modifyitems(config, items):
    # the small-size parity tests first, then the guard-band bounds checks,
    # then the full-size checks (the longest), so that a stopped run (-x)
    # still reports the parity of every kernel
    # and the allocation-free entry point's file after everything else
    def order(it):
        if "test_zz_no_alloc" in it.nodeid:
            return 3
        return 1 if "test_gpu_canaries" in it.nodeid else 2 if "test_gpu_fullsize" in it.nodeid else 0
    items.sort(key=order)
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
