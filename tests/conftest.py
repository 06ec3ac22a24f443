import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the libhatt kernels)")
    config.addinivalue_line("markers", "slow: larger CPU oracle cases")


def read_kat(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            ctr, key, out = (part.split() for part in line.split("|"))
            rows.append(([int(v, 16) for v in ctr], [int(v, 16) for v in key],
                         [int(v, 16) for v in out]))
    return rows


@pytest.fixture
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")
