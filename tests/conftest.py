import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size case (minutes)")


def pytest_sessionstart(session):
    # native crashes: dump every thread's Python stack to a file when asked
    path = os.environ.get("JN_FAULT_LOG")
    if path:
        import faulthandler
        fh = open(path, "w")
        session.config._jn_fault_file = fh
        faulthandler.enable(file=fh, all_threads=True)
