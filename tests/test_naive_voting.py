"""Naive voting (Algorithm 1) as written in oracle/naive.py, pinned against brute-force
depth (tests/brute.py, numpy in the global surface form) and against the generalized
voting of the oracle (Algorithm 2)."""
import numpy as np
import pytest

import brute
import oracle
from oracle.naive import naive_voting
from paper_2107_11810_gb300 import inputs

CASES = [
    ("line", lambda: inputs.line2d(n=300, inlier_frac=0.3, eps=0.02, seed=3)),
    ("plane", lambda: inputs.plane3d(n=120, inlier_frac=0.3, eps=0.08, sigma=0.002, seed=3)),
    ("pose", lambda: inputs.pose3dof(n=200, inlier_frac=0.3, eps_xy=2.0, eps_yaw_deg=4.0, noise_deg=0.05, seed=3)),
    ("rays", lambda: inputs.rays3d(n=300, inlier_frac=0.3, eps=0.03, noise=0.002, seed=3)),
    ("points", lambda: inputs.pointset2d(m=14, eps=0.16, noise=0.002, seed=3)),
    ("affine", lambda: inputs.affine4d(n=150, inlier_frac=0.3, eps=0.15, noise=0.005, seed=3)),
    ("pose6", lambda: inputs.pose6dof(n=40, inlier_frac=0.3, levels=2, seed=3)),
    ("radial", lambda: inputs.radial5dof(n=40, inlier_frac=0.3, levels=2, seed=3)),
]


@pytest.mark.parametrize("name,mk", CASES)
def test_votes_bounded_by_brute_force_and_generalized_depth(name, mk):
    p = mk()
    r = naive_voting(p.family, p.eps, p.bounds, p.params)
    lv = oracle.levels(p.family, p.eps, p.bounds)
    assert r["evaluations"] == p.n * int(np.prod([2 ** int(x) for x in lv["Lj"][: p.k]]))
    assert r["votes"] > 0
    # every counted surface is within half a leaf width (<= eps/2) of the cell's centre
    assert r["votes"] <= brute.depth(p.family, p.params, p.eps[p.k:], r["center"][None])[0]
    assert r["votes"] <= oracle.solve(p.family, p.eps, p.bounds, p.params)["depth"]


def test_noise_free_planted_lines_give_half_their_inliers_to_one_cell():
    rng = np.random.default_rng(4)
    for m, b in [(0.3125, 0.4375), (-0.7, 1.3), (0.05, -0.4)]:
        x = rng.uniform(0, 1, 64)
        params = np.stack([x, m * x + b])
        r = naive_voting(inputs.LINE2D, [0.01, 0.01], [-1, 1, -1, 2], params)
        # at the free cell holding m the 64 values span at most one leaf width of b
        assert r["votes"] >= 32
