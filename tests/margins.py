"""Sampled checks of the oracle's margin functions against the surface equations.

The surface-box test and the canonization error bound (Sec. 3.2) rest on three
margin functions of the oracle, and a mistake in any of them can leave every
brute-force pin green (it only moves a margin).  These helpers check each one
against the family's surface equation, evaluated here with numpy's sin/cos in
the global (textbook) form -- never through the oracle's own arithmetic:

* sigma_m(h): bound on |psi_m(x) - psi_m(c)| over a cell of half-widths h, psi_m
  the basis function that multiplies essential parameter t_m in F (it sets the
  essential-parameter snap step and the per-level rounding error);
* Lambda_ji(t): bound on the slope of F_j in free coordinate i, so that
  |F_j(x; t) - F_j(c; t)| <= sum_i Lambda_ji(t) h_i over a cell (the free-coordinate
  term of the surface-box radius);
* A_{l+1}: the accumulated canonization error, so that the canonical record of a
  surface after the level-l snap stays within A_{l+1} of the original surface over
  the whole level-l cell.

Sample points are drawn uniformly in each cell, plus its corners and the
midpoints of its edges (where a smooth function's change over a box peaks).
"""
from __future__ import annotations

import itertools

import numpy as np

import brute
import oracle

LINE2D, PLANE3D_SPH, POSE3DOF, POSE6DOF, RAYS3D, POINTSET2D, AFFINE4D, RADIAL5DOF, POSE7DOF = range(1, 10)


def _rot(x):
    from scipy.spatial.transform import Rotation
    sh = x.shape[:-1]
    return Rotation.from_rotvec(x.reshape(-1, 3)).as_matrix().reshape(sh + (3, 3))


def basis(family: int, x: np.ndarray) -> np.ndarray:
    """psi_m(x) [..., le] at free coordinates x [..., k]: the functions multiplying
    the essential parameters in each surface equation.  For POSE6DOF, where one
    parameter multiplies different functions in the x and y equations, [..., 2 le]:
    the x equation's functions, then the y equation's."""
    if family == LINE2D:            # b = y - x m: t = x multiplies -m
        return x[..., 0:1].copy()
    if family == PLANE3D_SPH:       # d = q . n(theta, phi)
        th, ph = x[..., 0], x[..., 1]
        return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=-1)
    if family == POSE3DOF:          # (x, y) = w - R(yaw) (a, b)
        return np.stack([np.cos(x[..., 0]), np.sin(x[..., 0])], axis=-1)
    if family == RAYS3D:            # y = a x + b, z = c x + d: a and c multiply x
        return np.concatenate([x[..., 0:1], x[..., 0:1]], axis=-1)
    if family == AFFINE4D:          # b = x4 - sum_i x_i a_i: t_i multiplies -a_i
        return -x[..., 0:3].copy()
    if family == POINTSET2D:        # a = g_a - u c - v d, b = g_b - v c + u d; t = (u, v)
        c, d = x[..., 0:1], x[..., 1:2]
        return np.concatenate([-c, -d, d, -c], axis=-1)
    if family == POSE6DOF:          # t = (w, xi w, eta w, xi, eta); rows of R(phi) and z
        Rm = _rot(x[..., 0:3])
        z = x[..., 3:4]
        zero3, zero1 = np.zeros(x.shape[:-1] + (3,)), np.zeros(x.shape[:-1] + (1,))
        fx = np.concatenate([-Rm[..., 0, :], Rm[..., 2, :], zero3, z, zero1], axis=-1)
        fy = np.concatenate([-Rm[..., 1, :], zero3, Rm[..., 2, :], zero1, z], axis=-1)
        return np.concatenate([fx, fy], axis=-1)
    if family == POSE7DOF:          # as POSE6DOF with r3 / f and z / f (free coords phi, z, f)
        Rm = _rot(x[..., 0:3])
        z, f = x[..., 3:4], x[..., 4:5]
        zero3, zero1 = np.zeros(x.shape[:-1] + (3,)), np.zeros(x.shape[:-1] + (1,))
        r3f = Rm[..., 2, :] / f
        fx = np.concatenate([-Rm[..., 0, :], r3f, zero3, z / f, zero1], axis=-1)
        fy = np.concatenate([-Rm[..., 1, :], zero3, r3f, zero1, z / f], axis=-1)
        return np.concatenate([fx, fy], axis=-1)
    if family == RADIAL5DOF:        # t = (rho w, w, rho): x = rho w . r1 - w . r2 - rho y
        Rm = _rot(x[..., 0:3])
        return np.concatenate([Rm[..., 0, :], -Rm[..., 1, :], -x[..., 3:4]], axis=-1)
    raise ValueError(family)


def t_part(family: int, t: np.ndarray, x: np.ndarray) -> np.ndarray:
    """The part of F_j(x; t) [..., d-k] that depends on t (the additive parameters
    cancel in every difference taken here)."""
    psi = basis(family, x)
    if family == LINE2D:
        return -(t[0] * psi[..., 0])[..., None]
    if family == PLANE3D_SPH:
        return (psi @ np.asarray(t))[..., None]
    if family == POSE3DOF:
        a, b = t
        c, s = psi[..., 0], psi[..., 1]
        return np.stack([-(a * c - b * s), -(a * s + b * c)], axis=-1)
    if family == RAYS3D:
        return np.stack([t[0] * psi[..., 0], t[1] * psi[..., 1]], axis=-1)
    if family == POINTSET2D:
        t = np.asarray(t, float)
        return np.stack([psi[..., :2] @ t, psi[..., 2:] @ t], axis=-1)
    if family == AFFINE4D:
        return (psi @ np.asarray(t, float))[..., None]
    if family in (POSE6DOF, POSE7DOF):
        t = np.asarray(t, float)
        return np.stack([psi[..., :11] @ t, psi[..., 11:] @ t], axis=-1)
    if family == RADIAL5DOF:
        return (psi @ np.asarray(t, float))[..., None]
    raise ValueError(family)


def cell_points(center: np.ndarray, h: np.ndarray, n: int, rng) -> np.ndarray:
    """n uniform points of the closed box center +- h, its corners and edge midpoints."""
    k = len(center)
    u = rng.uniform(-1.0, 1.0, size=(n, k))
    extra = np.array(list(itertools.product(*[(-1.0, 0.0, 1.0)] * k)))
    return center + np.concatenate([u, extra]) * h


def cell_center(lo, h, coords):
    return lo + (2 * np.asarray(coords, float) + 1) * h


def random_cell(Lj, level, rng):
    return np.array([int(rng.integers(0, 2 ** min(level, int(Lj[j])))) for j in range(len(Lj))])


def check_sigma(p, cells_per_level=4, points=100_000, seed=0, lib=None):
    """max over sampled cells of |psi(x) - psi(c)| / sigma(h), per level (must be <= 1)."""
    rng = np.random.default_rng(seed)
    lv = oracle.levels(p.family, p.eps, p.bounds, lib=lib)
    lo, k = p.bounds[0::2], p.k
    worst = []
    for l in range(lv["L"]):
        sig = oracle.sigma(p.family, lv["h"][l], bounds=p.bounds, lib=lib)
        if p.family in (POSE6DOF, POSE7DOF, POINTSET2D):
            sig = np.concatenate([sig, sig])          # the two dependent equations' functions
        w = 0.0
        for _ in range(cells_per_level):
            ci = random_cell(lv["Lj"], l, rng)
            c = cell_center(lo, lv["h"][l], ci)[:k]
            x = cell_points(c, lv["h"][l][:k], points, rng)
            dpsi = np.abs(basis(p.family, x) - basis(p.family, c[None])).max(axis=0)
            used = sig > 0
            assert np.all(dpsi[~used] == 0.0)
            w = max(w, float((dpsi[used] / sig[used]).max()))
        worst.append(w)
    return np.array(worst)


def check_lipschitz(p, ts, cells_per_level=3, points=100_000, seed=0, lib=None):
    """max over sampled cells and essential parameters t of
    |F(x; t) - F(c; t)| / (sum_i Lambda_ji(t) h_i), per level (must be <= 1), and of
    the same along each free coordinate alone: |F(c + u h_i e_i) - F(c)| /
    (Lambda_ji h_i) (so that a loose term cannot hide a missing one)."""
    rng = np.random.default_rng(seed)
    lv = oracle.levels(p.family, p.eps, p.bounds, lib=lib)
    lo, k = p.bounds[0::2], p.k
    worst = []
    for l in range(1, lv["L"] + 1):            # child cells: the radius uses their half-widths
        h = lv["h"][l]
        w = 0.0
        for _ in range(cells_per_level):
            ci = random_cell(lv["Lj"], l, rng)
            c = cell_center(lo, h, ci)[:k]
            x = cell_points(c, h[:k], points, rng)
            u = np.concatenate([np.linspace(-1.0, 1.0, 65), rng.uniform(-1.0, 1.0, 64)])
            for t in ts:
                lam = oracle.lipschitz(p.family, t, bounds=p.bounds, lib=lib)
                F0 = t_part(p.family, t, c[None])
                dF = np.abs(t_part(p.family, t, x) - F0).max(axis=0)
                bound = lam @ h[:k]
                w = max(w, float((dF / bound).max()))
                for i in range(k):                  # one free coordinate at a time
                    xi = np.repeat(c[None], len(u), axis=0)
                    xi[:, i] += u * h[i]
                    dFi = np.abs(t_part(p.family, t, xi) - F0).max(axis=0)
                    # a term that is linear in x_i meets its bound exactly: allow rounding
                    bi = lam[:, i] * h[i] * (1.0 + 1e-9) + 1e-12 * (1.0 + np.abs(F0[0]))
                    w = max(w, float((dFi / bi).max()))
        worst.append(w)
    return np.array(worst)


def surface_target(p, i, rng):
    """A point of the domain within eps/2 of original surface i (the surface passes
    through the leaf that contains it): random free coordinates, dependent
    coordinates on the surface plus a small offset.  None if it leaves the domain."""
    lo, hi = p.bounds[0::2], p.bounds[1::2]
    k = p.k
    for _ in range(50):
        x = lo[:k] + (hi[:k] - lo[:k]) * rng.uniform(size=k)
        pt = np.concatenate([x, np.zeros(p.d - k)])
        dep = -brute.vertical_residuals(p.family, p.params[:, i:i + 1], pt)[0, 0]
        dep = dep + rng.uniform(-0.5, 0.5, size=p.d - k) * p.eps[k:]
        if np.all(dep > lo[k:]) and np.all(dep < hi[k:]):
            return np.concatenate([x, dep])
    return None


def check_records(p, surfaces=30, points=2000, seed=0, lib=None):
    """For original surfaces and the root-to-leaf path through a point near each:
    (reached, worst) where reached = every surface reaches its leaf (the surface-box
    test never drops a surface that comes within eps of the cell), and worst = max
    over levels of |canonical - original| / A_{l+1} over the level-l cell (<= 1)."""
    rng = np.random.default_rng(seed)
    lv = oracle.levels(p.family, p.eps, p.bounds, lib=lib)
    L, lo, k = lv["L"], p.bounds[0::2], p.k
    W = p.bounds[1::2] - lo
    hL = lv["h"][L]
    reached, worst = True, 0.0
    for i in rng.choice(p.n, size=min(surfaces, p.n), replace=False):
        tgt = surface_target(p, int(i), rng)
        if tgt is None:
            continue
        leaf = np.minimum(np.floor((tgt - lo) / (2 * hL)).astype(np.int64), 2 ** lv["Lj"].astype(np.int64) - 1)
        f, t = oracle.path_records(p.family, p.eps, p.bounds, p.params, int(i), L, leaf, lib=lib)
        reached &= len(f) == L
        for l in range(len(f)):
            ci = np.array([leaf[j] >> (min(L, int(lv["Lj"][j])) - min(l, int(lv["Lj"][j]))) for j in range(p.d)])
            c = cell_center(lo, lv["h"][l], ci)
            x = cell_points(c[:k], lv["h"][l][:k], points, rng)
            # original surface: dependent value F(x; pi_i) in global form
            pts = np.concatenate([x, np.zeros((len(x), p.d - k))], axis=1)
            orig = -brute.vertical_residuals(p.family, p.params[:, i:i + 1], pts)[:, 0, :]
            # canonical record: value c_dep + f at the centre, moved by its own t-part
            canon = c[k:] + f[l] + (t_part(p.family, t[l], x) - t_part(p.family, t[l], c[None, :k]))
            dev = np.abs(orig - canon).max(axis=0)
            worst = max(worst, float((dev / lv["A"][l + 1]).max()))
    assert W.min() > 0
    return bool(reached), worst
