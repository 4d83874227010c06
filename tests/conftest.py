import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libhhg.so")
    config.addinivalue_line("markers", "slow: larger oracle cases")


def pytest_sessionfinish(session, exitstatus):
    """Under the bounds-checking library (HHG_LIBRARY=checked), a failed
    device-side index check reported when a mesh was closed -- including by
    the garbage collector, where it cannot raise -- fails the session."""
    if os.environ.get("HHG_LIBRARY") != "checked":
        return
    import gc
    gc.collect()
    hhg = sys.modules.get("paper_1805_10167_gb300.hhg")
    if hhg is not None and hhg.BOUNDS_FAILURES:
        print("\nindex checks failed:\n  " + "\n  ".join(hhg.BOUNDS_FAILURES), file=sys.stderr)
        session.exitstatus = 1
