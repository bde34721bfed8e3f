"""Planted mistakes in the oracle (on the CPU) must be caught by the pins.

A mistake that only tightens a conservative margin (for example dropping the
canonization error A from the UB radius, or shrinking one Lipschitz term that
the others dominate) changes a result only for surfaces within that margin of a
decision, which random instances rarely produce.  Such mistakes are caught by
the margin pins (tests/margins.py: sigma, Lambda and the accumulated error A
checked against the surface equations on the workloads' level structures) and,
for lines, by the exact-rational pin (tests/test_oracle_exact_line.py).

Each mutant is a copy of oracle/gv_oracle.c with one plausible mistake -- a
dropped term, a wrong sign, a wrong index, a transposed operand -- compiled
separately.  For each, at least one pin of tests/test_oracle_pins.py fails:
the reported depth drops below the brute-force depth at some point (lower
side), or exceeds the depth at the relaxed radius / counts a surface outside it
(upper side).
"""
import numpy as np
import pytest

import brute
import margins
import oracle
from paper_2107_11810_gb300 import inputs

MUTANTS = {
    "plane_sign": ("(f[0] + ((t[0] * g->dpsi[0] + t[1] * g->dpsi[1]) + t[2] * g->dpsi[2]))",
                   "(f[0] + ((t[0] * g->dpsi[0] + t[1] * g->dpsi[1]) - t[2] * g->dpsi[2]))"),
    "pose_index": ("fo[1] = (f[1] - (t[0] * g->dpsi[1] + t[1] * g->dpsi[0]))",
                   "fo[1] = (f[1] - (t[0] * g->dpsi[0] + t[1] * g->dpsi[1]))"),
    "line_residual_sign": ("fo[0] = (f[0] - t[0] * g->dpsi[0]) - g->shift[1];",
                           "fo[0] = (f[0] + t[0] * g->dpsi[0]) - g->shift[1];"),
    "canon_error_not_accumulated": ("p->A[l + 1][j] = p->A[l][j] + delta;", "p->A[l + 1][j] = delta;"),
    "snap_step_too_coarse": ("p->s_t[l][m] = pow2_floor(epsp_min / ((double)(le + 1) * sigma[m]));",
                             "p->s_t[l][m] = pow2_floor(64.0 * epsp_min / ((double)(le + 1) * sigma[m]));"),
    "radius_parent_width": ("R = R + lam[j * p->k + i] * p->h[l + 1][i];", "R = R + lam[j * p->k + i] * p->h[l + 1][i] * 0.25;"),
    "child_shift_sign": ("g->shift[j] = bit ? p->h[l + 1][j] : -p->h[l + 1][j];",
                         "g->shift[j] = bit ? -p->h[l + 1][j] : p->h[l + 1][j];"),
    "pose_basis_swap": ("psi[0] = gvo_vcos(yaw);\n        psi[1] = gvo_vsin(yaw);",
                        "psi[0] = gvo_vsin(yaw);\n        psi[1] = gvo_vcos(yaw);"),
    # margin-only mistakes (the brute-force pins alone let these through)
    "plane_sigma_without_phi": ("sigma[0] = h[0] + h[1];\n        sigma[1] = h[0] + h[1];",
                                "sigma[0] = h[0];\n        sigma[1] = h[0] + h[1];"),
    "plane_lipschitz_phi_from_qz": ("lam[1] = sqrt(t[0] * t[0] + t[1] * t[1]);",
                                    "lam[1] = fabs(t[2]);"),
    "pose_lipschitz_max_component": ("lam[0] = r;\n        lam[1] = r;",
                                     "lam[0] = fmax(fabs(t[0]), fabs(t[1]));\n        lam[1] = lam[0];"),
    "rays_residual_slope": ("fo[1] = (f[1] + t[1] * g->dpsi[0]) - g->shift[2];",
                            "fo[1] = (f[1] + t[0] * g->dpsi[0]) - g->shift[2];"),
    "rays_lipschitz_one_slope": ("dz/dx = c */\n        lam[0] = fabs(t[0]);\n        lam[1] = fabs(t[1]);",
                                 "dz/dx = c */\n        lam[0] = fabs(t[0]);\n        lam[1] = fabs(t[0]);"),
    "points_residual_sign": ("fo[1] = (f[1] - (t[1] * g->dpsi[0] - t[0] * g->dpsi[1])) - g->shift[3];",
                             "fo[1] = (f[1] - (t[1] * g->dpsi[0] + t[0] * g->dpsi[1])) - g->shift[3];"),
    "points_sigma_one_axis": ("sigma[0] = h[0] > h[1] ? h[0] : h[1];", "sigma[0] = h[1] * 0.5;"),
    "affine_residual_index": ("+ t[2] * g->dpsi[2])) - g->shift[3];", "+ t[2] * g->dpsi[1])) - g->shift[3];"),
    "affine_sigma_one_axis": ("sigma[2] = h[2];\n        break;", "sigma[2] = h[0] * 0.25;\n        break;"),
    "pose6_residual_row": ("double sy2 = (t[0] * d[3] + t[1] * d[4]) + t[2] * d[5];",
                           "double sy2 = (t[0] * d[0] + t[1] * d[1]) + t[2] * d[2];"),
    "pose6_rotation_sign": ("R[1] = b0 * ph[1] - a2;", "R[1] = b0 * ph[1] + a2;"),
    "pose6_lipschitz_without_w": ("double lx = nxw + nw, ly = nyw + nw;", "double lx = nxw, ly = nyw;"),
    "pose6_sigma_one_axis": ("double hr = (h[0] + h[1]) + h[2];", "double hr = h[0];"),
    "radial_residual_row": ("double s2 = (t[3] * d[3] + t[4] * d[4]) + t[5] * d[5];",
                            "double s2 = (t[3] * d[0] + t[4] * d[1]) + t[5] * d[2];"),
    "radial_lift_rho": ("double rho = eta / xi;", "double rho = xi / eta;"),
    "radial_lipschitz_without_w": ("double lx = nrw + nw;", "double lx = nrw;"),
    "radial_sigma_one_axis": ("double hphi = (h[0] + h[1]) + h[2];", "double hphi = h[2];"),
    "pose7_sigma_z_without_focal": ("double sz = h[3] / flo + (zmax * h[4]) * inv2;", "double sz = h[3] / flo;"),
    "pose7_lipschitz_focal_without_square": ("lam[4] = (nxw + fabs(t[9]) * zmax) * inv2;",
                                             "lam[4] = nxw + fabs(t[9]) * zmax;"),
    "pose7_lipschitz_z_without_focal": ("lam[3] = fabs(t[9]) / flo;", "lam[3] = fabs(t[9]);"),
    "pose7_basis_z_not_divided": ("psi[9] = z / f;", "psi[9] = z;"),
    "pose_sigma_halved": ("(a, b) */\n        sigma[0] = h[0];\n        sigma[1] = h[0];",
                          "(a, b) */\n        sigma[0] = 0.5 * h[0];\n        sigma[1] = 0.5 * h[0];"),
    "error_step_missing_essential_term": ("delta = delta + (p->s_t[l][m] * 0.5) * sigma[m];",
                                          "delta = delta + (p->s_t[l][m] * 0.25) * sigma[m];"),
}

CASES = {
    inputs.LINE2D: lambda s: inputs.line2d(n=300, inlier_frac=0.3, eps=0.02, seed=s),
    inputs.PLANE3D_SPH: lambda s: inputs.plane3d(n=120, inlier_frac=0.3, eps=0.08, sigma=0.002, seed=s),
    inputs.POSE3DOF: lambda s: inputs.pose3dof(n=200, inlier_frac=0.3, eps_xy=2.0, eps_yaw_deg=4.0,
                                               noise_deg=0.05, seed=s),
    inputs.POSE6DOF: lambda s: inputs.pose6dof(n=80, inlier_frac=0.3, levels=3, seed=s),
    inputs.RAYS3D: lambda s: inputs.rays3d(n=300, inlier_frac=0.3, eps=0.03, noise=0.002, seed=s),
    inputs.POINTSET2D: lambda s: inputs.pointset2d(m=14, eps=0.16, noise=0.002, seed=s),
    inputs.AFFINE4D: lambda s: inputs.affine4d(n=150, inlier_frac=0.3, eps=0.15, noise=0.005, seed=s),
    inputs.RADIAL5DOF: lambda s: inputs.radial5dof(n=80, inlier_frac=0.3, levels=3, seed=s),
    inputs.POSE7DOF: lambda s: inputs.pose7dof(n=60, inlier_frac=0.3, levels=3, seed=s),
}


def pins_hold(lib, fam, seed):
    """The level-structure, lower- and upper-side pins on one instance; False if any
    fails."""
    p = CASES[fam](seed)
    lv = oracle.levels(p.family, p.eps, p.bounds, lib=lib)
    L = lv["L"]
    # level structure: canonization error accumulates (strictly increasing) and stays
    # below eps/2; the essential-parameter steps respect their bound
    if not (np.all(np.diff(lv["A"], axis=0) > 0) and np.all(lv["A"][L] <= p.eps[p.k:] / 2 + 1e-12)):
        return False
    r = oracle.solve(p.family, p.eps, p.bounds, p.params, lib=lib)
    lo, W = p.bounds[0::2], p.bounds[1::2] - p.bounds[0::2]
    dep = p.eps[p.k:]
    rng = np.random.default_rng(seed)
    pts = np.concatenate([lo + W * rng.uniform(size=(3000, p.d)), p.truth[None]])
    grid = brute.leaf_centers(lo, W, lv["Lj"])
    best = max(int(brute.depth(p.family, p.params, dep, c).max()) for c in np.array_split(grid, max(1, len(grid) // 4096)))
    if r["depth"] < max(best, int(brute.depth(p.family, p.params, dep, pts).max())):
        return False
    L, hL = lv["L"], lv["h"][lv["L"]]
    st = lv["s_t"][-1].max()
    if p.family == inputs.LINE2D:
        free = (np.abs(p.params[0]).max() + st) * hL[: p.k].sum()
    elif p.family == inputs.PLANE3D_SPH:
        free = (np.linalg.norm(p.params, axis=0).max() + 2 * st) * hL[: p.k].sum()
    elif p.family == inputs.POSE3DOF:
        free = (np.hypot(p.params[2], p.params[3]).max() + 2 * st) * hL[: p.k].sum()
    elif p.family == inputs.RAYS3D:
        free = (np.maximum(np.abs(p.params[0]), np.abs(p.params[2])).max() + st) * hL[: p.k].sum()
    elif p.family == inputs.POINTSET2D:
        free = ((1.0 / np.hypot(p.params[0], p.params[1])).max() + st) * hL[: p.k].sum()
    elif p.family == inputs.AFFINE4D:
        free = (np.abs(p.params[0:3]).max() + st) * hL[: p.k].sum()
    elif p.family == inputs.POSE7DOF:
        flo, zmax = p.bounds[8], max(abs(p.bounds[6]), abs(p.bounds[7]))
        c = np.maximum(np.abs(p.params[3]), np.abs(p.params[4]))
        nw = np.linalg.norm(p.params[0:3], axis=0)
        free = ((((1.0 + c / flo) * nw).max() + 4 * st * (1.0 + 1.0 / flo)) * hL[0:3].sum()
                + (c.max() + st) / flo * hL[3] + ((c * (nw + zmax)).max() + 4 * st * (1.0 + zmax)) / flo ** 2 * hL[4])
    elif p.family == inputs.RADIAL5DOF:
        rho = np.abs(p.params[4] / p.params[3])
        free = ((((1.0 + rho) * np.linalg.norm(p.params[0:3], axis=0)).max() + 4 * st) * hL[0:3].sum()
                + (rho.max() + st) * hL[3])
    else:
        c = np.maximum(np.abs(p.params[3]), np.abs(p.params[4]))
        free = ((((1.0 + c) * np.linalg.norm(p.params[0:3], axis=0)).max() + 4 * st) * hL[0:3].sum()
                + (c.max() + st) * hL[3])
    ep = dep + hL[p.k:] + free + 2 * lv["A"][L] + 1e-9
    if r["depth"] > brute.depth(p.family, p.params, ep, r["best_point"][None])[0]:
        return False
    members = oracle.mask_to_indices(r["mask"], p.n)
    if len(members) != r["depth"]:
        return False
    res = brute.vertical_residuals(p.family, p.params[:, members], r["best_point"])[0]
    return bool(np.all(np.abs(res) <= ep))


MARGIN_CASES = {
    inputs.LINE2D: lambda: inputs.line2d(n=200, seed=inputs.SEED_BASE),
    inputs.PLANE3D_SPH: lambda: inputs.plane3d(n=200, seed=inputs.SEED_BASE + 1),
    inputs.POSE3DOF: lambda: inputs.pose3dof(n=200, seed=inputs.SEED_BASE + 2),
    inputs.POSE6DOF: lambda: inputs.pose6dof(n=200, seed=inputs.SEED_BASE + 4),
    inputs.RAYS3D: lambda: inputs.rays3d(n=200, seed=inputs.SEED_BASE + 5),
    inputs.POINTSET2D: lambda: inputs.pointset2d(m=15, seed=inputs.SEED_BASE + 6),
    inputs.AFFINE4D: lambda: inputs.affine4d(n=200, seed=inputs.SEED_BASE + 7),
    inputs.RADIAL5DOF: lambda: inputs.radial5dof(n=200, seed=inputs.SEED_BASE + 8),
    inputs.POSE7DOF: lambda: inputs.pose7dof(n=200, seed=inputs.SEED_BASE + 9),
}
MARGIN_T = {
    inputs.LINE2D: [np.array([1.0]), np.array([0.3])],
    inputs.PLANE3D_SPH: [np.array(v, float) for v in ([1, 1, 0], [0.2, 0.9, 0.4], [1, 1, 1])],
    inputs.POSE3DOF: [np.array(v, float) for v in ([50, 50], [-30, 80], [100, 0])],
    inputs.POSE6DOF: [np.array(v, float) for v in ([20, 20, 5, 20, 20, 5, -20, -20, -5, 1, -1],
                                                   [3, -14, 2, 1, -5, 0.5, 2, -9, 1, 0.4, 0.6])],
    inputs.RAYS3D: [np.array(v, float) for v in ([2, -2], [0.3, 1.7])],
    inputs.POINTSET2D: [np.array(v, float) for v in ([4, 0], [1.5, -2.5])],
    inputs.AFFINE4D: [np.array(v, float) for v in ([1, 1, 1], [0.2, -0.9, 0.5])],
    inputs.RADIAL5DOF: [np.array(v, float) for v in ([100, -60, 20, 20, -12, 4, 5],
                                                     [-3, 1.5, 0.6, 10, -5, 2, -0.3])],
    inputs.POSE7DOF: [np.array(v, float) for v in ([20, 20, 5, 20, 20, 5, -20, -20, -5, 1, -1],
                                                   [3, -14, 2, 1, -5, 0.5, 2, -9, 1, 0.4, 0.6])],
}


def margins_hold(lib, fam):
    """The margin pins (sigma, Lambda, accumulated error A) on the workload's level
    structure, with fewer samples than tests/test_oracle_margins.py; False if any fails."""
    p = MARGIN_CASES[fam]()
    if np.any(margins.check_sigma(p, cells_per_level=2, points=20_000, seed=1, lib=lib) > 1.0):
        return False
    if np.any(margins.check_lipschitz(p, MARGIN_T[fam], cells_per_level=2, points=5_000, seed=3, lib=lib)
              > 1.0 + 1e-12):
        return False
    reached, worst = margins.check_records(p, surfaces=25, points=1000, seed=4, lib=lib)
    return reached and worst <= 1.0


def test_unmodified_oracle_passes_the_pins():
    src = oracle.source()
    lib = oracle.load_variant(src, "identity")
    for fam in CASES:
        assert pins_hold(lib, fam, 1)
        assert margins_hold(lib, fam)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, name
    lib = oracle.load_variant(src.replace(old, new), name)
    caught = any(not margins_hold(lib, fam) for fam in CASES) or \
        any(not pins_hold(lib, fam, seed) for fam in CASES for seed in (1, 2, 3))
    assert caught, f"mutant {name} survived the pins"


@pytest.mark.parametrize("name", [m for m in sorted(MUTANTS) if m.startswith(("plane_sigma", "plane_lipschitz",
                                                                               "pose_lipschitz", "pose_sigma",
                                                                               "pose6_lipschitz", "pose6_sigma",
                                                                               "rays_lipschitz", "points_sigma", "affine_sigma",
                                                                               "radial_lipschitz", "radial_sigma",
                                                                               "pose7_sigma", "pose7_lipschitz",
                                                                               "error_step"))])
def test_margin_mistake_is_caught_by_the_margin_pins(name):
    old, new = MUTANTS[name]
    src = oracle.source()
    lib = oracle.load_variant(src.replace(old, new), name)
    assert any(not margins_hold(lib, fam) for fam in CASES), f"margin mutant {name} survived the margin pins"
