import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def libtnc():
    """Build (if stale) and load libtnc.so."""
    from paper_2205_00393_gb300 import build
    build.build_library()
    from paper_2205_00393_gb300 import _lib
    return _lib.load_library()
