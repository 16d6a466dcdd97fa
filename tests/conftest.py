import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_finish(session):
    """GPU tests of the public device API need the test-only user-kernel
    library: start its build now, so that it overlaps the other tests."""
    if any(("test_gpu_user_api" in item.nodeid or "test_gpu_trace" in item.nodeid) and item.get_closest_marker("gpu")
           for item in session.items):
        sys.path.insert(0, os.path.join(TESTS, "cuda"))
        import build_user
        build_user.start_background()
