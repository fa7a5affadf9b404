import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def load_golden(name):
    """Integer matrix fixture with a 'scale s' line: returns rows / s."""
    import numpy as np
    rows, scale = [], 1.0
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("scale"):
                scale = float(line.split()[1])
                continue
            rows.append([float(t) for t in line.split()])
    return np.array(rows) / scale
