import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


def load_golden(name):
    """Integer matrix fixture with a 'scale s' line: returns matrix / s."""
    scale = 1.0
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("scale"):
                scale = float(line.split()[1])
                continue
            rows.append([float(v) for v in line.split()])
    return np.array(rows) / scale


@pytest.fixture(scope="session")
def golden():
    return load_golden
