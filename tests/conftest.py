import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def load_golden_kernels():
    """Parse tests/golden/transfer_kernels.txt into {name: 3x3 float array}."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "transfer_kernels.txt")
    out, name, scale, rows = {}, None, None, []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("kernel"):
            _, name, scale = line.split()
            rows = []
            continue
        rows.append([float(v) for v in line.split()])
        if len(rows) == 3:
            out[name] = np.array(rows) / float(scale)
    return out
