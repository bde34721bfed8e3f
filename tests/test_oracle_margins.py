"""Pins of the oracle's margin functions (sigma, Lambda, accumulated error A).

The lower- and upper-side pins of tests/test_oracle_pins.py check results, and a
mistake that only tightens a conservative margin slips through them unless a
surface happens to sit inside that margin.  Here each margin is checked on its
own, against the surface equations (tests/margins.py), on the level structures
of the benchmark workloads (2D line eps 0.01, 3D plane eps 0.005, 3DoF camera
0.25 m / 0.5 deg, 6DoF camera with a +-30 deg rotation prior in a 10 m box, 7
levels, rays in the unit cube eps 0.002, point sets eps 0.01, affine hyperplanes in 4-space eps 0.01, the radial
camera with a +-30 deg rotation prior in a 10 m box, 7 levels, and the same with an unknown focal length in
[0.6, 1.3] of the true one):

* sigma_m bounds the change of every basis function across every level's cells
  (Sec. 3.2: the essential parameters are rounded to a step scaled by how much
  the surface can move across the box);
* Lambda bounds the change of F across a cell in the free coordinates (the
  "cell radius" part of the surface-box test, Sec. 3.2);
* after the snap at level l, every sampled original surface stays within A_{l+1}
  of its canonical record over the whole level-l cell (the accumulated rounding
  error that the eps update compensates, Sec. 3.2), and a surface that passes
  within eps/2 of a point reaches the leaf containing it.
"""
import math

import numpy as np
import pytest

import margins
from paper_2107_11810_gb300 import inputs

WORKLOADS = {
    "line": lambda: inputs.line2d(n=400, seed=inputs.SEED_BASE),
    "plane": lambda: inputs.plane3d(n=400, seed=inputs.SEED_BASE + 1),
    "pose": lambda: inputs.pose3dof(n=400, seed=inputs.SEED_BASE + 2),
    "pose6": lambda: inputs.pose6dof(n=400, seed=inputs.SEED_BASE + 4),
    "rays": lambda: inputs.rays3d(n=400, seed=inputs.SEED_BASE + 5),
    "points": lambda: inputs.pointset2d(m=20, seed=inputs.SEED_BASE + 6),
    "affine": lambda: inputs.affine4d(n=400, seed=inputs.SEED_BASE + 7),
    "radial": lambda: inputs.radial5dof(n=400, seed=inputs.SEED_BASE + 8),
    "pose7": lambda: inputs.pose7dof(n=400, seed=inputs.SEED_BASE + 9),
}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_sigma_bounds_the_basis_change_at_every_level(name):
    p = WORKLOADS[name]()
    worst = margins.check_sigma(p, cells_per_level=4, points=100_000, seed=1)
    assert np.all(worst <= 1.0), worst
    # and it is not vacuous: at the root the change reaches a fair part of the bound
    assert worst[0] > 0.3, worst


def essential_samples(p, rng):
    """Essential parameters of real surfaces plus adversarial directions."""
    if p.family == inputs.LINE2D:
        ts = [p.params[0, i:i + 1] for i in rng.choice(p.n, 20, replace=False)] + [np.array([1.0]), np.array([-1.0])]
    elif p.family == inputs.PLANE3D_SPH:
        ts = [p.params[:, i] for i in rng.choice(p.n, 20, replace=False)]
        ts += [np.array(v, float) for v in ([1, 1, 0], [1, 0, 0], [0, 0, 1], [0.7, -0.7, 0.1], [1, 1, 1])]
    elif p.family == inputs.POSE3DOF:
        ts = [p.params[2:, i] for i in rng.choice(p.n, 20, replace=False)]
        ts += [np.array(v, float) for v in ([50, 50], [-30, 80], [100, 0], [0, -100])]
    elif p.family == inputs.RAYS3D:
        ts = [p.params[[0, 2], i] for i in rng.choice(p.n, 20, replace=False)]
        ts += [np.array(v, float) for v in ([2, -2], [0, 1], [-1.5, 0])]
    elif p.family == inputs.AFFINE4D:
        ts = [p.params[0:3, i] for i in rng.choice(p.n, 20, replace=False)]
        ts += [np.array(v, float) for v in ([1, 1, 1], [1, -1, 0], [0, 0, 1])]
    elif p.family == inputs.POINTSET2D:         # t = p / |p|^2
        ts = []
        for i in rng.choice(p.n, 20, replace=False):
            px, py = p.params[0, i], p.params[1, i]
            ts.append(np.array([px, py]) / (px * px + py * py))
        ts += [np.array(v, float) for v in ([4, 0], [0, -4], [2.5, 2.5])]
    elif p.family == inputs.RADIAL5DOF:         # t = (rho w, w, rho), rho = eta / xi
        ts = []
        for i in rng.choice(p.n, 20, replace=False):
            w, rho = p.params[0:3, i], p.params[4, i] / p.params[3, i]
            ts.append(np.concatenate([rho * w, w, [rho]]))
        ts += [rng.normal(0.0, 10.0, 7) for _ in range(4)]
        ts += [np.array([100, -60, 20, 20, -12, 4, 5], float)]
    else:                      # 6DoF, 7DoF: t = (w, xi w, eta w, xi, eta), plus arbitrary coefficient vectors
        ts = []
        for i in rng.choice(p.n, 20, replace=False):
            w, xi, eta = p.params[0:3, i], p.params[3, i], p.params[4, i]
            ts.append(np.concatenate([w, xi * w, eta * w, [xi, eta]]))
        ts += [rng.normal(0.0, 10.0, 11) for _ in range(4)]
        ts += [np.array([20, 20, 5, 20, 20, 5, -20, -20, -5, 1, -1], float)]
    return ts


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_lipschitz_bounds_the_surface_change_over_child_cells(name):
    p = WORKLOADS[name]()
    ts = essential_samples(p, np.random.default_rng(2))
    worst = margins.check_lipschitz(p, ts, cells_per_level=3, points=20_000, seed=3)
    assert np.all(worst <= 1.0 + 1e-12), worst
    assert worst.max() > 0.5, worst


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_canonical_records_stay_within_accumulated_error(name):
    p = WORKLOADS[name]()
    reached, worst = margins.check_records(p, surfaces=40, points=3000, seed=4)
    assert reached
    assert worst <= 1.0, worst
    assert worst > 0.05, worst            # the bound is exercised, not vacuous


def test_plane_sigma_needs_its_phi_term():
    # n_x = sin(theta) cos(phi) moves by about h_phi across a cell at theta = phi = pi/2
    # (where its theta-derivative vanishes): a bound of h_theta alone is too small
    # for the workload's cells (h_phi = 2 h_theta); sigma covers it
    import oracle
    p = WORKLOADS["plane"]()
    h = np.array([1e-3, 2e-3, 1e-3])
    sig = oracle.sigma(p.family, h)
    c = np.array([math.pi / 2, math.pi / 2])
    x = margins.cell_points(c, h[:2], 20_000, np.random.default_rng(5))
    d = np.abs(margins.basis(p.family, x) - margins.basis(p.family, c[None])).max(axis=0)
    assert np.all(d <= sig)
    assert d[0] > 1.9 * h[0]
