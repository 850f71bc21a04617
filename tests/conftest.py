import os
import sys
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running case")


def load_golden(name: str) -> dict:
    """Parse a fixture under tests/golden: 'key value...' lines, '#' comments.
    Edges are 'u-v' or 'u-v:w'."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "edges":
                edges = []
                for tok in vals:
                    uv, _, w = tok.partition(":")
                    u, v = uv.split("-")
                    edges.append((int(u), int(v), int(w) if w else 1))
                out[key] = edges
            elif key in ("q", "q_start"):
                out[key] = Fraction(vals[0])
            elif key in ("partition", "iter1"):
                out[key] = [int(x) for x in vals]
            elif key == "optimal":
                out[key] = vals[0] == "yes"
            else:
                out[key] = int(vals[0])
    return out


@pytest.fixture
def golden():
    return load_golden
