import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running statistical case")


_RECORD = {}


@pytest.fixture(scope="session")
def record():
    """record(name, value): a measured error or statistic kept for the
    precision statement; written as JSON to $PARITY_RECORD at the end of the
    session when that variable is set."""
    def put(name, value):
        _RECORD[name] = value
    return put


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("PARITY_RECORD")
    if path and _RECORD:
        import json
        with open(path, "w") as fh:
            json.dump(_RECORD, fh, indent=1, sort_keys=True)
