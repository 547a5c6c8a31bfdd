import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def load_matrix(name):
    """Read a golden matrix file: '#' comment lines, a 'scale a/b' line, integer rows."""
    import numpy as np
    from fractions import Fraction
    rows, scale = [], 1.0
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("scale"):
                tok = line.split()[1]
                scale = float(Fraction(tok)) if "k" not in tok else tok
                continue
            rows.append([int(v) for v in line.split()])
    return np.array(rows, dtype=np.float64), scale


def paper_value(key):
    with open(os.path.join(GOLDEN, "paper_values.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == key:
                return float(parts[1])
    raise KeyError(key)


def cpu_threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count() or 1
