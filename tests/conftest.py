import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libbridges.so")
    config.addinivalue_line("markers", "slow: large inputs (minutes)")


def load_golden(name):
    """Parses a tests/golden fixture: returns (u, v, V, expected (k,2) array)."""
    lines = [ln.strip() for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    V = int(lines[0].split()[1])
    m = int(lines[1].split()[1])
    edges = np.array([[int(x) for x in ln.split()] for ln in lines[2:2 + m]], dtype=np.int32).reshape(m, 2)
    k = int(lines[2 + m].split()[1])
    exp = np.array([[int(x) for x in ln.split()] for ln in lines[3 + m:3 + m + k]], dtype=np.int32).reshape(k, 2)
    return edges[:, 0].copy(), edges[:, 1].copy(), V, exp


def load_golden_cuts(name):
    """The fixture's hand-derived cut vertices (its optional `cuts k` section after the bridges),
    as a sorted int32 array, or None if the fixture has none."""
    lines = [ln.strip() for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    at = [i for i, ln in enumerate(lines) if ln.split()[0] == "cuts"]
    if not at:
        return None
    k = int(lines[at[0]].split()[1])
    return np.array([int(ln) for ln in lines[at[0] + 1:at[0] + 1 + k]], dtype=np.int32)


def golden_names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))


@pytest.fixture(scope="session")
def cuda_lib():
    """The CUDA path's binding; skips when no GPU is visible."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_07346_gb300 as pb
    pb.load()
    return pb
