import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU and the built liblsas library")
    config.addinivalue_line(
        "markers", "slow: statistical or full-size checks that take longer")


def pytest_collection_modifyitems(config, items):
    # tests that need a GPU are skipped, not failed, on a machine without one,
    # unless they were selected explicitly with -m gpu
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    markexpr = config.getoption("-m") or ""
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords and "gpu" not in markexpr.replace("not gpu", ""):
            it.add_marker(skip)
