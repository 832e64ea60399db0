import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def golden_lines(name):
    """Non-comment, non-empty lines of a golden fixture, split into tokens."""
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line)
    return out


def parse_points(text):
    return np.array([[int(v) for v in p.split()] for p in text.split(";")], dtype=np.int64)


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.build()
    return O
