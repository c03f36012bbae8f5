import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def read_golden(name):
    """Parse 'key: a/b c/d ...' lines of a golden fixture into {key: [floats]}."""
    from fractions import Fraction
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, vals = line.split(":", 1)
            out[key.strip()] = [float(Fraction(v)) for v in vals.split()]
    return out
