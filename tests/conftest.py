import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library's Python binding, built in-tree; fails loudly if it cannot load."""
    import paper_1710_01133_gb300 as fabm
    fabm.load()
    return fabm


_PARITY = []


@pytest.fixture
def parity(request):
    """check(err, bar, label=''): assert a measured error against its bar and
    record it; with FABM_PARITY_REPORT set, the session writes every record
    (test, label, err, bar) to that JSON file."""
    def check(err, bar, label=""):
        _PARITY.append({"test": request.node.name, "label": str(label),
                        "err": float(err), "bar": float(bar)})
        assert err <= bar, (label, err, bar)
    return check


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("FABM_PARITY_REPORT")
    if path and _PARITY:
        with open(path, "w") as fh:
            json.dump(_PARITY, fh, indent=1)
