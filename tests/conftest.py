import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session", autouse=True)
def _build_oracle():
    import oracle
    oracle.build()
    yield


GOLDEN = os.path.join(ROOT, "tests", "golden")


def read_golden(name):
    """Non-comment, non-empty lines of tests/golden/<name>."""
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]


def golden_patterns():
    """{(name, phase): set of (r, c)} from tests/golden/patterns.txt."""
    out = {}
    for ln in read_golden("patterns.txt"):
        head, cells = ln.split(":")
        name, phase = head.split()
        out[(name, int(phase))] = {tuple(int(v) for v in rc.split(",")) for rc in cells.split()}
    return out
