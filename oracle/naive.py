"""Naive voting (Algorithm 1) for every family (test infrastructure only: only
``tests/`` may import this module).

The paper's baseline: iterate the k free coordinates on an eps-grid, compute the
d - k dependent values of every surface there from the surface equations (Sec. 3,
Eq. 1, in global form), and tally one vote per surface for the d-cell those values
fall in; the answer is the cell with the most votes.  Here the eps-grid is the leaf
grid of the search (its cells are at most eps wide in every coordinate) and the free
coordinates are taken at the leaf centres.  Its work is n surface evaluations per
free cell, which is the operation count the paper compares with the predicate calls
of generalized voting (Sec. 4.2.5).

Pins (tests/test_naive_voting.py): the best cell's votes never exceed the brute-force
depth at its centre, nor the generalized voting's depth (a counted surface lies within
half a leaf width, at most eps/2, of the cell's centre in every dependent coordinate);
noise-free planted lines give at least half their inliers to one cell; the number of
evaluations is n times the number of free cells.
"""
from __future__ import annotations

import itertools

import numpy as np
import torch

from . import FAMILY_SHAPE, levels
from .softscore import residuals


def dependent_values(family: int, params: np.ndarray, x_free: np.ndarray) -> np.ndarray:
    """F(x_free; pi_i) [n, d-k] of every surface at one point of the free coordinates
    (the residual at a point whose dependent coordinates are 0, negated)."""
    d, k, _, _ = FAMILY_SHAPE[family]
    p = torch.zeros(d, dtype=torch.float64)
    p[:k] = torch.as_tensor(x_free, dtype=torch.float64)
    return -residuals(family, torch.from_numpy(np.ascontiguousarray(params, dtype=np.float64)), p).numpy()


def naive_voting(family: int, eps, bounds, params: np.ndarray) -> dict:
    """Algorithm 1 on the leaf grid: the best cell's votes, its integer leaf
    coordinates, its centre, and the number of surface evaluations."""
    d, k, _, _ = FAMILY_SHAPE[family]
    lv = levels(family, eps, bounds)
    bounds = np.asarray(bounds, dtype=np.float64)
    lo, hi = bounds[0::2], bounds[1::2]
    Lj = lv["Lj"]
    w = (hi - lo) / 2.0 ** Lj                        # leaf widths
    n = params.shape[1]
    best, best_cell = -1, None
    evals = 0
    for ci in itertools.product(*[range(2 ** int(Lj[j])) for j in range(k)]):
        xc = lo[:k] + (np.array(ci) + 0.5) * w[:k]
        F = dependent_values(family, params, xc)
        evals += n
        b = np.floor((F - lo[k:]) / w[k:]).astype(np.int64)
        ok = np.all((b >= 0) & (b < 2 ** Lj[k:].astype(np.int64)), axis=1)
        if not ok.any():
            continue
        keys, counts = np.unique(b[ok], axis=0, return_counts=True)
        i = int(np.argmax(counts))                   # ties: the first (smallest) key
        if counts[i] > best:
            best, best_cell = int(counts[i]), np.concatenate([np.array(ci), keys[i]])
    if best_cell is None:
        return dict(votes=0, cell=None, center=None, evaluations=evals)
    return dict(votes=best, cell=best_cell, center=lo + (best_cell + 0.5) * w, evaluations=evals)
