import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libgoat")
    config.addinivalue_line("markers", "slow: long-running")


def read_golden(name):
    """Parse a golden text fixture: '#' comments, 'matrix' block, 'key v1 v2 ...' lines."""
    out = {}
    rows = None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line == "matrix":
                rows = []
                out["matrix"] = rows
                continue
            parts = line.split()
            try:
                float(parts[0])
                is_num = True
            except ValueError:
                is_num = False
            if is_num and rows is not None:
                rows.append([float(x) for x in parts])
            else:
                rows = None
                out[parts[0]] = [float(x) for x in parts[1:]]
    return out


@pytest.fixture
def golden():
    return read_golden
