import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size case (minutes of CPU)")


def pytest_sessionstart(session):
    # FDAS_CHECKED=1: the binding loads the checked build of the library
    # (device bounds checks, workspace canaries) for every test
    if os.environ.get("FDAS_CHECKED") == "1":
        import importlib
        importlib.import_module("paper_2211_13517_gb300.build").build(checked=True)


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
