"""Golden fixtures (tests/golden/, written by tests/golden/make_golden.py from the
oracle): the oracle reproduces them, and so does the CUDA path (GPU)."""
import json
import os

import numpy as np
import pytest

import oracle
from golden.make_golden import CASES

# the fixtures tests/golden/make_golden.py writes (inputs stored with them)
FIXTURES = sorted(os.path.join(os.path.dirname(__file__), "golden", name + ".json") for name, _, _ in CASES)


class Fixture:
    def __init__(self, g):
        self.family = g["family"]
        self.eps = np.array([float.fromhex(x) for x in g["eps"]])
        self.bounds = np.array([float.fromhex(x) for x in g["bounds"]])
        self.params = np.array([[float.fromhex(x) for x in row] for row in g["params"]])
        self.n = self.params.shape[1]


def load(path):
    with open(path) as f:
        g = json.load(f)
    return g, Fixture(g)


def check(g, depth, leaf, point, mask):
    assert depth == g["depth"]
    assert [int(x) for x in leaf] == g["best_leaf"]
    assert [float(x).hex() for x in point] == g["best_point"]
    assert [int(w) for w in np.asarray(mask).view(np.uint32)] == g["mask"]


@pytest.mark.parametrize("path", FIXTURES, ids=[os.path.basename(f) for f in FIXTURES])
def test_oracle_reproduces_golden(path):
    g, p = load(path)
    r = oracle.solve(p.family, p.eps, p.bounds, p.params)
    check(g, r["depth"], r["best_leaf"], r["best_point"], r["mask"])


@pytest.mark.gpu
@pytest.mark.parametrize("path", FIXTURES, ids=[os.path.basename(f) for f in FIXTURES])
@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_reproduces_golden(path, precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11810_gb300 import build, vote
    build.build()
    g, p = load(path)
    s = vote.Solver(p.family, p.eps, p.bounds, precision=precision)
    r = s.solve(torch.from_numpy(p.params).cuda())
    check(g, r["depth"], r["best_leaf"], r["best_point"], vote.mask_words_to_numpy(r["mask"])[: (p.n + 31) // 32])
