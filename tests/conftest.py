import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def pytest_collection_modifyitems(config, items):
    # A file named test_zz_* is collected last by name; keep that order stable.
    items.sort(key=lambda it: (os.path.basename(str(it.fspath)).startswith("test_zz_"),))


_GPU = None


def _have_gpu():
    global _GPU
    if _GPU is None:
        try:
            import torch
            _GPU = bool(torch.cuda.is_available())
        except Exception:
            _GPU = False
    return _GPU


def pytest_runtest_setup(item):
    if item.get_closest_marker("gpu") is not None and not _have_gpu():
        pytest.skip("no CUDA device visible")
