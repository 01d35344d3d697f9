import ctypes
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes tens of seconds")


@pytest.fixture(scope="session")
def repo_root():
    return ROOT


def pytest_sessionfinish(session, exitstatus):
    """Under the bounds-checked library (MSC_LIB_VARIANT=check) write the library's index-check
    report to the file MSC_BOUNDS_REPORT names (read by test_gpu_bounds_check.py)."""
    path = os.environ.get("MSC_BOUNDS_REPORT")
    mod = sys.modules.get("paper_2609_39474_b300._lib")
    if not path or os.environ.get("MSC_LIB_VARIANT") != "check" or mod is None:
        return
    count, first = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    rc = mod.lib.msc_bounds_check_report(ctypes.byref(count), ctypes.byref(first), 0)
    with open(path, "w") as fh:
        json.dump({"rc": rc, "count": count.value, "first": first.value, "lib": mod.LIB_PATH}, fh)
