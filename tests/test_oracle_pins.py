"""Pins of the oracle against facts fixed by the paper and by the mathematics.

Every pin is independent of the oracle's own arithmetic: brute-force depth from
the global surface equations (tests/brute.py), the exact arrangement maximum for
lines, Algorithm 1 (naive voting), planted inliers, the approximation guarantee
implied by the Lipschitz test and the canonization error bound, invariance of the
result under pruning, visiting order and merging of canonical surfaces, and
special cases with known answers.
"""
import math

import mpmath
import numpy as np
import pytest

import brute
import oracle
from paper_2107_11810_gb300 import inputs

L2, PL, P3, P6, RY, PS, AF, RD, P7 = (oracle.LINE2D, oracle.PLANE3D_SPH, oracle.POSE3DOF, oracle.POSE6DOF,
                                      oracle.RAYS3D, oracle.POINTSET2D, oracle.AFFINE4D, oracle.RADIAL5DOF,
                                      oracle.POSE7DOF)


def small_plane(n, seed, eps=0.08, frac=0.3):
    p = inputs.plane3d(n=n, inlier_frac=frac, eps=eps, sigma=0.002, seed=seed)
    return p


def small_pose(n, seed, frac=0.3):
    p = inputs.pose3dof(n=n, inlier_frac=frac, eps_xy=2.0, eps_yaw_deg=4.0, noise_deg=0.05, seed=seed)
    return p


def small_line(n, seed, eps=0.01, frac=0.3):
    return inputs.line2d(n=n, inlier_frac=frac, eps=eps, seed=seed)


def small_pose6(n, seed, frac=0.3, levels=3):
    return inputs.pose6dof(n=n, inlier_frac=frac, levels=levels, seed=seed)


def small_rays(n, seed, frac=0.3, eps=0.03):
    return inputs.rays3d(n=n, inlier_frac=frac, eps=eps, noise=0.002, seed=seed)


def small_points(m, seed, eps=0.16):
    return inputs.pointset2d(m=m, eps=eps, noise=0.002, seed=seed)


def small_affine(n, seed, eps=0.15, frac=0.3):
    return inputs.affine4d(n=n, inlier_frac=frac, eps=eps, noise=0.005, seed=seed)


def small_radial(n, seed, frac=0.3, levels=3):
    return inputs.radial5dof(n=n, inlier_frac=frac, levels=levels, seed=seed)


def small_pose7(n, seed, frac=0.3, levels=3):
    return inputs.pose7dof(n=n, inlier_frac=frac, levels=levels, seed=seed)


CASES = [
    ("line", lambda s: small_line(300, s, eps=0.02)),
    ("plane", lambda s: small_plane(120, s)),
    ("pose", lambda s: small_pose(200, s)),
    ("pose6", lambda s: small_pose6(80, s)),
    ("rays", lambda s: small_rays(300, s)),
    ("points", lambda s: small_points(14, s)),
    ("affine", lambda s: small_affine(150, s)),
    ("radial", lambda s: small_radial(80, s)),
    ("pose7", lambda s: small_pose7(60, s)),
]


def dep_eps(p):
    return p.eps[p.k:]


# ---------------------------------------------------------------------------
# sin / cos of cell-centre angles
# ---------------------------------------------------------------------------

def test_vsin_vcos_within_one_ulp():
    mpmath.mp.prec = 200
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.uniform(-1.0, 7.0, 3000), np.linspace(0, 2 * math.pi, 513),
                         [0.0, math.pi / 4, math.pi / 2, math.pi, 3 * math.pi / 2, 2 * math.pi]])
    for x in xs:
        s_ref = float(mpmath.sin(mpmath.mpf(float(x))))
        c_ref = float(mpmath.cos(mpmath.mpf(float(x))))
        s, c = oracle.vsin(x), oracle.vcos(x)
        assert abs(s - s_ref) <= math.ulp(max(abs(s_ref), 2 ** -60)) * 1.0 + 1e-300, x
        assert abs(c - c_ref) <= math.ulp(max(abs(c_ref), 2 ** -60)) * 1.0 + 1e-300, x


# ---------------------------------------------------------------------------
# level structure
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,mk", CASES)
def test_levels_structure(name, mk):
    p = mk(1)
    lv = oracle.levels(p.family, p.eps, p.bounds)
    W = p.bounds[1::2] - p.bounds[0::2]
    L = lv["L"]
    # leaf width <= eps in every coordinate, and L_j is the smallest such level
    for j in range(p.d):
        assert 2 * lv["h"][L, j] <= p.eps[j]
        assert lv["Lj"][j] == 0 or W[j] * 2.0 ** (-(lv["Lj"][j] - 1)) > p.eps[j]
    # snap steps are powers of two; essential steps never shrink with depth
    for s in np.concatenate([lv["s_f"].ravel(), lv["s_t"].ravel()]):
        assert math.frexp(s)[0] == 0.5
    assert np.all(np.diff(lv["s_t"], axis=0) >= 0)
    # the accumulated canonization error stays below eps/2 (eps' = eps/L)
    assert np.all(lv["A"][L] <= dep_eps(p) / 2 + 1e-12)
    assert np.all(np.diff(lv["A"], axis=0) > 0)


# ---------------------------------------------------------------------------
# P1: lower side -- reported depth >= brute-force depth anywhere
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,mk", CASES)
@pytest.mark.parametrize("seed", [1, 2])
def test_reported_at_least_dense_grid_max(name, mk, seed):
    p = mk(seed)
    r = oracle.solve(p.family, p.eps, p.bounds, p.params)
    lv = oracle.levels(p.family, p.eps, p.bounds)
    lo = p.bounds[0::2]
    W = p.bounds[1::2] - p.bounds[0::2]
    grid = brute.leaf_centers(lo, W, lv["Lj"])
    best = 0
    for chunk in np.array_split(grid, max(1, len(grid) // 4096)):
        best = max(best, int(brute.depth(p.family, p.params, dep_eps(p), chunk).max()))
    assert r["depth"] >= best
    # and at random points of the domain
    rng = np.random.default_rng(seed)
    pts = lo + W * rng.uniform(size=(4000, p.d))
    assert r["depth"] >= brute.depth(p.family, p.params, dep_eps(p), pts).max()


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_line2d_reported_at_least_exact_arrangement_max(seed):
    p = small_line(60, seed, eps=0.05, frac=0.4)
    r = oracle.solve(p.family, p.eps, p.bounds, p.params)
    exact = brute.line2d_exact_max_depth(p.params, 0.05, p.bounds)
    assert r["depth"] >= exact
    assert r["depth"] >= brute.naive_voting_line2d(p.params, 0.05, p.bounds)


def test_line2d_config_reported_at_least_naive_voting():
    p = inputs.line2d()   # the 10,000-point line workload
    r = oracle.solve(p.family, p.eps, p.bounds, p.params)
    assert r["depth"] >= brute.naive_voting_line2d(p.params, 0.01, p.bounds)
    # planted line: every inlier is within eps (noise 0.002*sqrt(2) < eps)
    assert r["depth"] >= brute.depth(p.family, p.params, dep_eps(p), p.truth[None])[0] >= 1000


# ---------------------------------------------------------------------------
# P2: upper side -- every counted surface is within the relaxed radius
# ---------------------------------------------------------------------------

def relaxed_eps(p, lv):
    """eps+ = eps + h_L(dep) + Lambda_max * sum h_L(free) + 2 A_L (+ slack for the
    change of the Lipschitz factor by snapping)."""
    L = lv["L"]
    hL = lv["h"][L]
    st = lv["s_t"][-1].max()
    if p.family == L2:
        lam = np.abs(p.params[0]).max() + st
    elif p.family == PL:
        lam = np.linalg.norm(p.params, axis=0).max() + 2 * st
    elif p.family == P3:
        lam = np.hypot(p.params[2], p.params[3]).max() + 2 * st
    elif p.family == RY:
        lam = np.maximum(np.abs(p.params[0]), np.abs(p.params[2])).max() + st
    elif p.family == PS:       # |u| = |v| bound: 1/|p|
        lam = (1.0 / np.hypot(p.params[0], p.params[1])).max() + st
    elif p.family == AF:       # |db/da_i| = |x_i| <= 1
        lam = np.abs(p.params[0:3]).max() + st
    elif p.family == P7:       # as 6DoF with 1/f: |dF/dphi_a| <= (1 + c/f_lo) |w|, |dF/dz| <= c/f_lo,
        # |dF/df| <= c (|w| + z_max)/f_lo^2, c = max(|xi|, |eta|)
        flo = p.bounds[8]
        zmax = max(abs(p.bounds[6]), abs(p.bounds[7]))
        c = np.maximum(np.abs(p.params[3]), np.abs(p.params[4]))
        nw = np.linalg.norm(p.params[0:3], axis=0)
        lam_phi = ((1.0 + c / flo) * nw).max() + 4 * st * (1.0 + 1.0 / flo)
        lam_z = (c.max() + st) / flo
        lam_f = ((c * (nw + zmax)).max() + 4 * st * (1.0 + zmax)) / flo ** 2
        return (dep_eps(p) + hL[p.k:] + lam_phi * hL[0:3].sum() + lam_z * hL[3] + lam_f * hL[4]
                + 2 * lv["A"][L] + 1e-9)
    elif p.family == RD:       # |dx/dphi_a| <= (1 + |rho|) |w|, |dx/dy| = |rho|, rho = eta / xi
        rho = np.abs(p.params[4] / p.params[3])
        lam_phi = ((1.0 + rho) * np.linalg.norm(p.params[0:3], axis=0)).max() + 4 * st
        lam_y = rho.max() + st
        return dep_eps(p) + hL[p.k:] + lam_phi * hL[0:3].sum() + lam_y * hL[3] + 2 * lv["A"][L] + 1e-9
    else:          # |dF/dphi_a| <= (1 + max(|xi|, |eta|)) |w|, |dF/dz| <= max(|xi|, |eta|)
        c = np.maximum(np.abs(p.params[3]), np.abs(p.params[4]))
        lam_phi = ((1.0 + c) * np.linalg.norm(p.params[0:3], axis=0)).max() + 4 * st
        lam_z = c.max() + st
        return dep_eps(p) + hL[p.k:] + lam_phi * hL[0:3].sum() + lam_z * hL[3] + 2 * lv["A"][L] + 1e-9
    free = hL[: p.k].sum()
    return dep_eps(p) + hL[p.k:] + lam * free + 2 * lv["A"][L] + 1e-9


@pytest.mark.parametrize("name,mk", CASES)
@pytest.mark.parametrize("seed", [1, 2])
def test_reported_at_most_relaxed_depth_and_mask(name, mk, seed):
    p = mk(seed)
    r = oracle.solve(p.family, p.eps, p.bounds, p.params)
    lv = oracle.levels(p.family, p.eps, p.bounds)
    ep = relaxed_eps(p, lv)
    assert r["depth"] <= brute.depth(p.family, p.params, ep, r["best_point"][None])[0]
    members = oracle.mask_to_indices(r["mask"], p.n)
    assert len(members) == r["depth"]
    # every member lies within the relaxed radius of the reported point
    res = brute.vertical_residuals(p.family, p.params[:, members], r["best_point"])[0]
    assert np.all(np.abs(res) <= ep)
    # every surface within eps of the reported point is a member
    close = brute.inlier_set(p.family, p.params, dep_eps(p), r["best_point"])
    assert np.all(np.isin(close, members))


# ---------------------------------------------------------------------------
# P4: planted inliers
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,mk", CASES)
def test_planted_lower_bound(name, mk):
    p = mk(7)
    r = oracle.solve(p.family, p.eps, p.bounds, p.params)
    assert r["depth"] >= brute.depth(p.family, p.params, dep_eps(p), p.truth[None])[0]
    assert r["depth"] >= 0.5 * len(p.inliers)


# ---------------------------------------------------------------------------
# P5-P7: structural invariants, pruning/order/merging invariance
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,mk", CASES)
def test_invariance_prune_order_merge(name, mk):
    p = mk(3)
    ref = oracle.solve(p.family, p.eps, p.bounds, p.params)
    for flags in (oracle.NO_PRUNE, oracle.REVERSE, oracle.NO_MERGE, oracle.NO_MERGE | oracle.REVERSE):
        r = oracle.solve(p.family, p.eps, p.bounds, p.params, flags=flags, members=True)
        assert r["depth"] == ref["depth"], flags
        assert np.array_equal(r["best_leaf"], ref["best_leaf"]), flags
        assert np.array_equal(r["mask"], ref["mask"]), flags
        if flags & oracle.NO_MERGE:
            # members tracked directly through the recursion == replayed mask
            assert np.array_equal(r["members"], oracle.mask_to_indices(ref["mask"], p.n))
    # merging does reduce the work somewhere
    a = oracle.solve(p.family, p.eps, p.bounds, p.params)["stats"][0]
    b = oracle.solve(p.family, p.eps, p.bounds, p.params, flags=oracle.NO_MERGE)["stats"][0]
    assert a <= b


@pytest.mark.parametrize("name,mk", CASES)
def test_trace_counts_equal_replay_and_monotone(name, mk):
    p = mk(4)
    r = oracle.solve(p.family, p.eps, p.bounds, p.params, flags=oracle.NO_PRUNE, trace_cap=200000)
    tr = r["trace"]
    assert np.all(tr["lb"] <= tr["ub"])
    lv = oracle.levels(p.family, p.eps, p.bounds)
    Lj = lv["Lj"]
    ub_of = {(int(l), tuple(c)): int(u) for l, c, u in zip(tr["level"], tr["coords"], tr["ub"])}
    ub_of[(0, (0,) * p.d)] = p.n
    for (l, c), u in list(ub_of.items())[:5000]:
        if l == 0:
            continue
        parent = tuple(ci >> (1 if l - 1 < Lj[j] else 0) for j, ci in enumerate(c))
        assert u <= ub_of[(l - 1, parent)]
    rng = np.random.default_rng(0)
    for x in rng.choice(len(tr["ub"]), size=min(25, len(tr["ub"])), replace=False):
        ub, lb = oracle.cell_counts(p.family, p.eps, p.bounds, p.params, tr["level"][x], tr["coords"][x])
        assert (ub, lb) == (tr["ub"][x], tr["lb"][x])


# ---------------------------------------------------------------------------
# P8: special cases
# ---------------------------------------------------------------------------

def test_empty_input():
    for mk in (lambda: small_line(10, 1), lambda: small_plane(10, 1), lambda: small_pose(10, 1),
               lambda: small_pose6(10, 1), lambda: small_rays(10, 1), lambda: small_points(3, 1),
               lambda: small_affine(10, 1), lambda: small_radial(10, 1), lambda: small_pose7(10, 1)):
        p = mk()
        r = oracle.solve(p.family, p.eps, p.bounds, p.params[:, :0])
        assert r["depth"] == 0
        assert np.all(r["best_leaf"] == 0)


def test_identical_surfaces():
    p = small_line(50, 2)
    params = np.repeat(p.params[:, :1], 37, axis=1)
    r = oracle.solve(p.family, p.eps, p.bounds, params)
    assert r["depth"] == 37
    assert oracle.mask_to_indices(r["mask"], 37).size == 37
    s = oracle.solve(p.family, p.eps, p.bounds, params, flags=oracle.NO_MERGE)
    assert r["stats"][0] * 10 < s["stats"][0]       # one canonical record per cell


def test_noise_free_line_depth_n():
    rng = np.random.default_rng(5)
    m, b = 0.3125, 0.4375
    x = rng.uniform(0, 1, 80)
    params = np.stack([x, m * x + b])
    r = oracle.solve(L2, [0.01, 0.01], [-1, 1, -1, 2], params)
    assert r["depth"] == 80
    # the leaf containing the planted (m, b) is reached by every surface
    lv = oracle.levels(L2, [0.01, 0.01], [-1, 1, -1, 2])
    L, hL = lv["L"], lv["h"][lv["L"]]
    leaf = [int((m + 1) / (2 * hL[0])), int((b + 1) / (2 * hL[1]))]
    assert oracle.cell_counts(L2, [0.01, 0.01], [-1, 1, -1, 2], params, L, leaf)[0] == 80
    # ties go to the lexicographically smallest leaf
    assert tuple(r["best_leaf"]) <= tuple(leaf)


def test_eps_covers_domain_returns_everything():
    p = small_line(40, 3)
    r = oracle.solve(L2, [5.0, 5.0], [-1, 1, -1, 2], p.params)
    assert r["depth"] == 40
    assert np.all(r["best_leaf"] == 0)


def test_invalid_inputs_rejected():
    p = small_line(10, 1)
    with pytest.raises(ValueError):
        oracle.solve(L2, [0.0, 0.01], p.bounds, p.params)
    with pytest.raises(ValueError):
        oracle.solve(L2, p.eps, [1, -1, -1, 2], p.params)
    bad = p.params.copy()
    bad[0, 3] = np.nan
    with pytest.raises(ValueError):
        oracle.solve(L2, p.eps, p.bounds, bad)


# ---------------------------------------------------------------------------
# the multi-core oracle (CPU baseline) gives the serial oracle's results
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,mk", CASES)
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_parallel_oracle_equals_serial(name, mk, threads):
    p = mk(6)
    a = oracle.solve(p.family, p.eps, p.bounds, p.params)
    b = oracle.solve_parallel(p.family, p.eps, p.bounds, p.params, threads=threads)
    assert b["depth"] == a["depth"]
    assert np.array_equal(b["best_leaf"], a["best_leaf"])
    assert np.array_equal(b["best_point"], a["best_point"])
    assert np.array_equal(b["mask"], a["mask"])
    assert b["stats"][4] == threads
