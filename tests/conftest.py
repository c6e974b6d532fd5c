import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (runs the CUDA library through its C ABI)")
    config.addinivalue_line(
        "markers", "slow: long CPU test (still part of the default suite)")


@pytest.fixture(scope="session")
def eik_lib():
    """The CUDA library, built in-tree if needed (GPU tests only)."""
    from paper_1306_4743_gb300 import eik
    return eik.load()
