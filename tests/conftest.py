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
    config.addinivalue_line(
        "markers", "fmm_solution(name, arg): needs the oracle FMM of a large workload "
                   "(started in the background after collection, tests/_oracle_jobs.py)")


def pytest_collection_finish(session):
    tasks = []
    for item in session.items:
        for m in item.iter_markers("fmm_solution"):
            tasks.append(tuple(m.args))
    if not tasks:
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except Exception:
        return
    from tests import _oracle_jobs
    _oracle_jobs.start(tasks)


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("tests._oracle_jobs")
    if mod is not None:
        mod.stop()


@pytest.fixture(scope="session")
def eik_lib():
    """The CUDA library, built in-tree if needed (GPU tests only)."""
    from paper_1306_4743_gb300 import eik
    return eik.load()
