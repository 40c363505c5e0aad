import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (the CUDA library's parity and property tests)")
    config.addinivalue_line("markers", "slow: longer CPU runs of the oracle")
    config.addinivalue_line("markers", "full: the named configurations at full size and step count "
                                       "(minutes; run with LBM_FULL_CONFIGS=1)")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if os.environ.get("LBM_FULL_CONFIGS") != "1":
        skip_full = pytest.mark.skip(reason="full-size configurations: set LBM_FULL_CONFIGS=1")
        for it in items:
            if "full" in it.keywords:
                it.add_marker(skip_full)
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
