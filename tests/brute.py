"""Brute-force depth evaluation, written from the surface equations alone.

These helpers evaluate ``depth_eps(p) = #{i : |p_dep - F(p_free; pi_i)| <= eps}``
directly from the original match parameters with numpy's sin/cos, in the
textbook (global) form of each surface -- not in the local, snapped frame the
oracle uses.  They pin the oracle (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import itertools

import numpy as np

LINE2D, PLANE3D_SPH, POSE3DOF, POSE6DOF, RAYS3D, POINTSET2D, AFFINE4D, RADIAL5DOF, POSE7DOF = range(1, 10)


def vertical_residuals(family: int, params: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Residuals [npts, n, d-k] of every surface at every point (global form)."""
    pts = np.atleast_2d(np.asarray(pts, float))
    if family == LINE2D:                 # b = y - x m      (Sec. 3, Eq. 2)
        x, y = params
        m, b = pts[:, 0:1], pts[:, 1:2]
        return (b - (y[None, :] - x[None, :] * m))[..., None]
    if family == PLANE3D_SPH:            # d = q . n(theta, phi)   (Sec. 4.1)
        qx, qy, qz = params
        th, ph, dd = pts[:, 0:1], pts[:, 1:2], pts[:, 2:3]
        nx, ny, nz = np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)
        return (dd - (qx * nx + qy * ny + qz * nz))[..., None]
    if family == POSE3DOF:               # camera position given yaw
        w1, w2, a, b = params
        yaw, x, y = pts[:, 0:1], pts[:, 1:2], pts[:, 2:3]
        fx = w1 - (a * np.cos(yaw) - b * np.sin(yaw))
        fy = w2 - (a * np.sin(yaw) + b * np.cos(yaw))
        return np.stack([x - fx, y - fy], axis=-1)
    if family == AFFINE4D:               # hyperplane x4 = a . x + b in dual form (Sec. 4.1)
        x = np.asarray(params[0:3], float)
        return (pts[:, 3:4] - (params[3][None, :] - pts[:, 0:3] @ x))[..., None]
    if family == POINTSET2D:             # (a, b) solving q = [[a, b], [-b, a]] p + (c, d) (Sec. 4.4)
        px, py, qx, qy = params
        c, d, a, b = pts[:, 0:1], pts[:, 1:2], pts[:, 2:3], pts[:, 3:4]
        n2 = px * px + py * py
        sa = (px * (qx - c) + py * (qy - d)) / n2
        sb = (py * (qx - c) - px * (qy - d)) / n2
        return np.stack([a - sa, b - sb], axis=-1)
    if family == RAYS3D:                 # y = a x + b, z = c x + d (Sec. 4.3)
        a, b, c, d = params
        x, y, z = pts[:, 0:1], pts[:, 1:2], pts[:, 2:3]
        return np.stack([y - (a * x + b), z - (c * x + d)], axis=-1)
    if family == POSE6DOF:               # calibrated camera: X = R(phi) w + (x, y, z) (Sec. 4.2.3)
        from scipy.spatial.transform import Rotation
        w = np.asarray(params[0:3], float)                    # [3, n]
        xi, eta = params[3], params[4]
        Rm = Rotation.from_rotvec(pts[:, 0:3]).as_matrix()    # [npts, 3, 3]
        Rw = np.einsum("pij,jn->pin", Rm, w)                  # rows r_i . w: [npts, 3, n]
        z, x, y = pts[:, 3:4], pts[:, 4:5], pts[:, 5:6]
        depth_ = Rw[:, 2, :] + z
        fx = xi[None, :] * depth_ - Rw[:, 0, :]
        fy = eta[None, :] * depth_ - Rw[:, 1, :]
        return np.stack([x - fx, y - fy], axis=-1)
    if family == POSE7DOF:               # unknown focal: f (X_1, X_2) / X_3 = (xi, eta) (Sec. 4.2.2)
        from scipy.spatial.transform import Rotation
        w = np.asarray(params[0:3], float)
        xi, eta = params[3], params[4]
        Rm = Rotation.from_rotvec(pts[:, 0:3]).as_matrix()
        Rw = np.einsum("pij,jn->pin", Rm, w)
        z, f, x, y = pts[:, 3:4], pts[:, 4:5], pts[:, 5:6], pts[:, 6:7]
        depth_ = Rw[:, 2, :] + z
        fx = xi[None, :] * depth_ / f - Rw[:, 0, :]
        fy = eta[None, :] * depth_ / f - Rw[:, 1, :]
        return np.stack([x - fx, y - fy], axis=-1)
    if family == RADIAL5DOF:             # radial camera rows (r1, -y), (r2, x) (Sec. 4.2.4)
        from scipy.spatial.transform import Rotation
        w = np.asarray(params[0:3], float)
        xi, eta = params[3], params[4]
        Rm = Rotation.from_rotvec(pts[:, 0:3]).as_matrix()
        Rw = np.einsum("pij,jn->pin", Rm, w)
        y, x = pts[:, 3:4], pts[:, 4:5]
        fx = eta[None, :] * (Rw[:, 0, :] - y) / xi[None, :] - Rw[:, 1, :]
        return (x - fx)[..., None]
    raise ValueError(family)


def depth(family: int, params: np.ndarray, eps_dep, pts, rel_tol: float = 0.0) -> np.ndarray:
    """depth_eps at each point (L-infinity over the dependent coordinates)."""
    r = vertical_residuals(family, params, pts)
    e = np.asarray(eps_dep, float) * (1.0 + rel_tol)
    return np.all(np.abs(r) <= e, axis=-1).sum(axis=1)


def inlier_set(family: int, params: np.ndarray, eps_dep, pt) -> np.ndarray:
    r = vertical_residuals(family, params, np.asarray(pt, float)[None, :])[0]
    return np.nonzero(np.all(np.abs(r) <= np.asarray(eps_dep, float), axis=-1))[0]


def leaf_centers(lo, W, Lj, level=None):
    """All cell centres at a level (default: the leaf level)."""
    Lj = np.asarray(Lj)
    L = int(Lj.max()) if level is None else level
    axes = []
    for j in range(len(Lj)):
        e = min(L, int(Lj[j]))
        h = W[j] * 2.0 ** (-(e + 1))
        axes.append(lo[j] + (2 * np.arange(2 ** e) + 1) * h)
    return np.array(list(itertools.product(*axes)))


def line2d_exact_max_depth(params: np.ndarray, eps: float, bounds) -> int:
    """Exact maximum over the closed domain of depth_eps for the dual lines
    b = y_i - x_i m: the maximum of a piecewise-constant count over an
    arrangement of the 2n lines b = y_i - x_i m +- eps is attained at one of its
    vertices, at an intersection with the domain edges m = lo/hi, or at a corner."""
    x, y = params
    mlo, mhi, blo, bhi = bounds
    slopes = np.concatenate([-x, -x])
    icpt = np.concatenate([y - eps, y + eps])
    cand = [(mlo, blo), (mlo, bhi), (mhi, blo), (mhi, bhi)]
    for s, c in zip(slopes, icpt):
        for m in (mlo, mhi):
            b = c + s * m
            if blo <= b <= bhi:
                cand.append((m, b))
        for b in (blo, bhi):
            if s != 0:
                m = (b - c) / s
                if mlo <= m <= mhi:
                    cand.append((m, b))
    nl = len(slopes)
    for i in range(nl):
        ds = slopes[i] - slopes[i + 1:]
        dc = icpt[i + 1:] - icpt[i]
        ok = ds != 0
        m = dc[ok] / ds[ok]
        b = icpt[i] + slopes[i] * m
        sel = (m >= mlo) & (m <= mhi) & (b >= blo) & (b <= bhi)
        cand.extend(zip(m[sel], b[sel]))
    cand = np.array(cand)
    best = 0
    for chunk in np.array_split(cand, max(1, len(cand) // 2000)):
        best = max(best, int(depth(LINE2D, params, [eps], chunk, rel_tol=1e-9).max()))
    return best


def naive_voting_line2d(params: np.ndarray, eps: float, bounds) -> int:
    """Naive voting (Algorithm 1): iterate the free coordinate on an eps-grid,
    compute each surface's dependent value there and tally votes per eps-cell of
    the dependent coordinate.  Returns the best cell's count; every surface in a
    cell lies within eps (the cell width) of its centre, so the count is a lower
    bound on the max depth."""
    x, y = params
    mlo, mhi, blo, bhi = bounds
    best = 0
    for m in np.arange(mlo, mhi + 1e-12, eps):
        b = y - x * m
        cell = np.floor((b - blo) / eps).astype(np.int64)
        ok = (b >= blo) & (b <= bhi)
        if ok.any():
            best = max(best, int(np.bincount(cell[ok]).max()))
    return best
