import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle():
    from oracle import Oracle
    return Oracle()


@pytest.fixture(scope="session")
def tiny():
    from paper_1910_05200_gb300 import synthetic as S
    return S.make_workload("tiny", seed=0)


def pytest_sessionfinish(session, exitstatus):
    """With FACERT_PARITY_LOG set, write every parity check's measured errors
    (tests/parity.py RECORD) to that file, one JSON object per line."""
    path = os.environ.get("FACERT_PARITY_LOG")
    if not path:
        return
    try:
        from tests.parity import RECORD
    except ImportError:
        return
    import json
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    with open(path, "w") as f:
        for row in RECORD:
            f.write(json.dumps(row) + "\n")
