"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws scenes and writes them as surface-parameter arrays; it
holds none of the voting arithmetic.  Both the CUDA path and the CPU oracle read
the arrays it returns.  Every generator is ``numpy.random.default_rng(seed)``
(PCG64); the standard workloads use seed ``2107118100 + i`` for workload ``i``.

Surface parameters are FP64, structure-of-arrays ``params[P, n]``:

* ``LINE2D``      (Sec. 3, Eq. 2; line fitting of Sec. 4.1):  P = 2, rows (x, y) of the
  image points; voting space (m, b) with the dual line b = y - x m.
* ``PLANE3D_SPH`` (Sec. 4.1, hyperplanes in d-space, in spherical form): P = 3,
  rows (qx, qy, qz); voting space (theta, phi, d) with d = q . n(theta, phi).
* ``POSE3DOF``    (camera posing with known gravity, focal length and height; the
  3DoF reduction of the 5DoF surfaces of Sec. 4.2.1): P = 4, rows (w1, w2, a, b);
  voting space (yaw, x, y) with x = w1 - (a cos yaw - b sin yaw) and
  y = w2 - (a sin yaw + b cos yaw); (a, b) = r (cos beta, sin beta), r the
  horizontal distance implied by the elevation, beta the bearing azimuth.
* ``POSE6DOF``    (calibrated camera, Sec. 4.2.3: the 7DoF surfaces of Sec. 4.2.2
  with f = 1): P = 5, rows (w1, w2, w3, xi, eta) of a match between world point w
  and normalized image point (xi, eta); voting space (phi1, phi2, phi3, z, x, y),
  phi the axis-angle vector of the rotation and (x, y, z) the translation of the
  camera frame X = R(phi) w + (x, y, z), with x = xi (r3 . w + z) - r1 . w and
  y = eta (r3 . w + z) - r2 . w.
* ``RAYS3D``      (intersection of rays in 3-space, Sec. 4.3): P = 4, rows (a, b, c, d)
  of the ray y = a x + b, z = c x + d; voting space (x, y, z).
* ``POINTSET2D``  (point-set similarity alignment, Sec. 4.4): P = 4, rows (px, py, qx, qy)
  of a hypothetical correspondence p -> q under q_x = a p_x + b p_y + c,
  q_y = -b p_x + a p_y + d; voting space (c, d, a, b).
* ``AFFINE4D``    (hyperplane fitting in the affine form, Sec. 4.1, d = 4): P = 4, rows
  (x1, x2, x3, x4) of points; voting space (a1, a2, a3, b) with the dual hyperplane
  b = x4 - (a1 x1 + a2 x2 + a3 x3).
* ``RADIAL5DOF``  (radial camera, unknown focal length, Sec. 4.2.4): P = 5, rows
  (w1, w2, w3, xi, eta) of a match between world point w and image point (xi, eta);
  voting space (phi1, phi2, phi3, y, x) of the radial camera with rows
  (r1, -y) and (r2, x), where eta (r1 . w - y) = xi (r2 . w + x), i.e.
  x = eta (r1 . w - y) / xi - r2 . w.
* ``POSE7DOF``    (camera posing with unknown focal length, Sec. 4.2.2): P = 5, rows
  (w1, w2, w3, xi, eta) as for 6DoF; voting space (phi1, phi2, phi3, z, f, x, y) with
  x = xi (r3 . w + z) / f - r1 . w and y = eta (r3 . w + z) / f - r2 . w.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LINE2D, PLANE3D_SPH, POSE3DOF, POSE6DOF, RAYS3D, POINTSET2D, AFFINE4D, RADIAL5DOF, POSE7DOF = range(1, 10)
FAMILY_NAMES = {LINE2D: "LINE2D", PLANE3D_SPH: "PLANE3D_SPH", POSE3DOF: "POSE3DOF", POSE6DOF: "POSE6DOF",
                RAYS3D: "RAYS3D", POINTSET2D: "POINTSET2D", AFFINE4D: "AFFINE4D", RADIAL5DOF: "RADIAL5DOF",
                POSE7DOF: "POSE7DOF"}
FAMILY_DK = {LINE2D: (2, 1), PLANE3D_SPH: (3, 2), POSE3DOF: (3, 1), POSE6DOF: (6, 4), RAYS3D: (3, 1),
             POINTSET2D: (4, 2), AFFINE4D: (4, 3), RADIAL5DOF: (5, 4), POSE7DOF: (7, 5)}
SEED_BASE = 2107118100


@dataclass
class Problem:
    family: int
    eps: np.ndarray          # [d]
    bounds: np.ndarray       # [2d]: lo0, hi0, lo1, hi1, ...
    params: np.ndarray       # [P, n] float64 (SoA)
    truth: np.ndarray        # [d] planted solution in voting coordinates
    inliers: np.ndarray      # indices of planted inliers
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.params.shape[1])

    @property
    def d(self) -> int:
        return FAMILY_DK[self.family][0]

    @property
    def k(self) -> int:
        return FAMILY_DK[self.family][1]


# ---------------------------------------------------------------------------
# 2D line fitting
# ---------------------------------------------------------------------------

def line2d(n: int = 10_000, inlier_frac: float = 0.10, eps: float = 0.01, noise: float = 0.002,
           seed: int = SEED_BASE + 0, quantize: int | None = None) -> Problem:
    """Points in [0,1]^2: ``inlier_frac`` of them within uniform +-noise
    (perpendicular) of a random line y = m x + b (m ~ U[-1,1], b ~ U[0,1]), the
    rest uniform.  Voting domain m in [-1, 1], b in [-1, 2].

    ``quantize=q`` rounds coordinates to multiples of 2^-q (dyadic inputs)."""
    rng = np.random.default_rng(seed)
    m = rng.uniform(-1.0, 1.0)
    b = rng.uniform(0.0, 1.0)
    n_in = int(round(n * inlier_frac))
    pts = np.empty((n, 2))
    got = 0
    while got < n_in:
        x0 = rng.uniform(0.0, 1.0, size=2 * (n_in - got) + 8)
        u = rng.uniform(-noise, noise, size=x0.size)
        nrm = 1.0 / math.sqrt(1.0 + m * m)
        px = x0 - u * m * nrm
        py = m * x0 + b + u * nrm
        ok = (px >= 0) & (px <= 1) & (py >= 0) & (py <= 1)
        take = np.stack([px[ok], py[ok]], axis=1)[: n_in - got]
        pts[got:got + len(take)] = take
        got += len(take)
    pts[n_in:] = rng.uniform(0.0, 1.0, size=(n - n_in, 2))
    perm = rng.permutation(n)
    pts = pts[perm]
    inliers = np.nonzero(perm < n_in)[0]
    if quantize is not None:
        pts = np.round(pts * 2.0 ** quantize) / 2.0 ** quantize
    return Problem(LINE2D, np.array([eps, eps]), np.array([-1.0, 1.0, -1.0, 2.0]),
                   np.ascontiguousarray(pts.T), np.array([m, b]), inliers, "line2d",
                   dict(inlier_frac=inlier_frac, noise=noise))


# ---------------------------------------------------------------------------
# 3D plane fitting, (theta, phi, d) parameter space
# ---------------------------------------------------------------------------

def plane3d(n: int = 1_000_000, inlier_frac: float = 0.02, eps: float = 0.005, sigma: float = 0.001,
            seed: int = SEED_BASE + 1) -> Problem:
    """Points in the unit cube: ``inlier_frac`` on a random plane (normal uniform on
    the sphere, through a U[0,1]^3 point) plus N(0, sigma) along the normal, the
    rest uniform.  Voting domain theta in [0, pi], phi in [0, 2 pi],
    d in [-sqrt 3, sqrt 3]; eps_d = eps, eps_theta = eps_phi = eps / sqrt 3."""
    rng = np.random.default_rng(seed)
    while True:
        v = rng.normal(size=3)
        nrm = v / np.linalg.norm(v)
        p0 = rng.uniform(0.0, 1.0, size=3)
        dd = float(nrm @ p0)
        corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float)
        s = corners @ nrm - dd
        if s.min() < -0.05 and s.max() > 0.05:
            break
    theta = math.acos(max(-1.0, min(1.0, nrm[2])))
    phi = math.atan2(nrm[1], nrm[0]) % (2 * math.pi)
    n_in = int(round(n * inlier_frac))
    pts = np.empty((n, 3))
    got = 0
    while got < n_in:
        q = rng.uniform(0.0, 1.0, size=(2 * (n_in - got) + 8, 3))
        q = q - np.outer(q @ nrm - dd, nrm)
        ok = np.all((q >= 0) & (q <= 1), axis=1)
        q = q[ok][: n_in - got]
        q = q + np.outer(rng.normal(0.0, sigma, size=len(q)), nrm)
        pts[got:got + len(q)] = q
        got += len(q)
    pts[n_in:] = rng.uniform(0.0, 1.0, size=(n - n_in, 3))
    perm = rng.permutation(n)
    pts = pts[perm]
    inliers = np.nonzero(perm < n_in)[0]
    r3 = math.sqrt(3.0)
    e_ang = eps / r3
    return Problem(PLANE3D_SPH, np.array([e_ang, e_ang, eps]),
                   np.array([0.0, math.pi, 0.0, 2 * math.pi, -r3, r3]),
                   np.ascontiguousarray(pts.T), np.array([theta, phi, dd]), inliers, "plane3d",
                   dict(inlier_frac=inlier_frac, sigma=sigma))


# ---------------------------------------------------------------------------
# 3DoF camera voting (known gravity, focal length and camera height)
# ---------------------------------------------------------------------------

def pose3dof(n: int = 1_000_000, inlier_frac: float = 0.01, eps_xy: float = 0.25,
             eps_yaw_deg: float = 0.5, noise_deg: float = 0.1, box=(100.0, 100.0, 10.0),
             seed: int = SEED_BASE + 2, rng: np.random.Generator | None = None) -> Problem:
    """3D points uniform in ``box``; a camera at (x, y) ~ U[0, box_x] x U[0, box_y],
    yaw ~ U[0, 2 pi), height h ~ U[1, 9].  Inlier matches carry the true bearing
    with N(0, noise) on azimuth and elevation; outliers pair a random point with a
    random bearing (uniform direction).  Matches with |elevation| < 1 deg are
    redrawn.  Each match becomes (w1, w2, a, b) with r = (w3 - h) / tan(elev),
    a = r cos(beta), b = r sin(beta), beta the azimuth relative to the heading.
    Voting domain yaw in [0, 2 pi], x in [0, box_x], y in [0, box_y]."""
    if rng is None:
        rng = np.random.default_rng(seed)
    bx, by, bz = box
    cam = np.array([rng.uniform(0, bx), rng.uniform(0, by)])
    yaw = rng.uniform(0, 2 * math.pi)
    h = rng.uniform(1.0, 9.0)
    n_in = int(round(n * inlier_frac))
    min_el = math.radians(1.0)
    sig = math.radians(noise_deg)
    out = np.empty((4, n))

    def draw_points(m):
        return np.stack([rng.uniform(0, bx, m), rng.uniform(0, by, m), rng.uniform(0, bz, m)], axis=1)

    got = 0
    while got < n_in:
        m = 2 * (n_in - got) + 8
        w = draw_points(m)
        dx, dy, dz = w[:, 0] - cam[0], w[:, 1] - cam[1], w[:, 2] - h
        rho = np.hypot(dx, dy)
        beta = np.arctan2(dy, dx) - yaw + rng.normal(0, sig, m)
        el = np.arctan2(dz, rho) + rng.normal(0, sig, m)
        ok = (np.abs(el) >= min_el) & (rho > 1e-3)
        w, beta, el = w[ok][: n_in - got], beta[ok][: n_in - got], el[ok][: n_in - got]
        r = (w[:, 2] - h) / np.tan(el)
        sl = slice(got, got + len(w))
        out[0, sl], out[1, sl] = w[:, 0], w[:, 1]
        out[2, sl], out[3, sl] = r * np.cos(beta), r * np.sin(beta)
        got += len(w)
    while got < n:
        m = 2 * (n - got) + 8
        w = draw_points(m)
        v = rng.normal(size=(m, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        el = np.arcsin(np.clip(v[:, 2], -1, 1))
        beta = np.arctan2(v[:, 1], v[:, 0])
        ok = np.abs(el) >= min_el
        w, beta, el = w[ok][: n - got], beta[ok][: n - got], el[ok][: n - got]
        r = (w[:, 2] - h) / np.tan(el)
        sl = slice(got, got + len(w))
        out[0, sl], out[1, sl] = w[:, 0], w[:, 1]
        out[2, sl], out[3, sl] = r * np.cos(beta), r * np.sin(beta)
        got += len(w)
    perm = rng.permutation(n)
    out = out[:, perm]
    inliers = np.nonzero(perm < n_in)[0]
    e_yaw = math.radians(eps_yaw_deg)
    return Problem(POSE3DOF, np.array([e_yaw, eps_xy, eps_xy]),
                   np.array([0.0, 2 * math.pi, 0.0, bx, 0.0, by]),
                   np.ascontiguousarray(out), np.array([yaw, cam[0], cam[1]]), inliers, "pose3dof",
                   dict(inlier_frac=inlier_frac, height=h))


def pose3dof_batch(num: int = 256, n_lo: float = 1e3, n_hi: float = 1e6, frac_lo: float = 0.005,
                   frac_hi: float = 0.05, seed: int = SEED_BASE + 3) -> list[Problem]:
    """``num`` independent 3DoF problems, n = round(10^U[log10 n_lo, log10 n_hi]) and
    inlier ratio ~ U[frac_lo, frac_hi]."""
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(num):
        n = int(round(10 ** rng.uniform(math.log10(n_lo), math.log10(n_hi))))
        frac = rng.uniform(frac_lo, frac_hi)
        probs.append(pose3dof(n=n, inlier_frac=frac, rng=rng))
    return probs


def rotvec_matrix(ph) -> np.ndarray:
    """Rotation matrix of an axis-angle vector (numpy's own trigonometry; scene
    generation only)."""
    ph = np.asarray(ph, float)
    th = float(np.linalg.norm(ph))
    if th == 0.0:
        return np.eye(3)
    k = ph / th
    K = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + math.sin(th) * K + (1.0 - math.cos(th)) * (K @ K)


def pose6dof(n: int = 5000, inlier_frac: float = 0.05, prior_deg: float = 30.0, box: float = 10.0,
             levels: int = 7, noise_deg: float = 0.1, points=(20.0, 20.0, 5.0), fov: float = 1.0,
             seed: int = SEED_BASE + 4, rng: np.random.Generator | None = None) -> Problem:
    """Calibrated-camera posing (6DoF).  World points uniform in
    [0, points_0] x [0, points_1] x [0, points_2]; the camera maps w to
    X = R(phi) w + t.  Truth: phi = phi_prior + U[-prior, prior]^3 with phi_prior
    uniform in the ball of radius 1 rad, t ~ U[0, box]^3 (redrawn until a quarter of
    the points lie in front of the camera).  Inliers: points with X_3 > 1 m seen at
    (X_1/X_3, X_2/X_3) within the field of view |xi|, |eta| <= fov, the bearing
    perturbed by N(0, noise) on both image angles; outliers: a random point with a
    random image point of the field of view.  Voting domain: phi in
    phi_prior +- prior per axis, (z, x, y) in [0, box]^3; every coordinate splits
    ``levels`` times (leaf widths 2 prior / 2^levels and box / 2^levels), and the
    depth tolerance of x and y is their leaf width (a constant vertical distance)."""
    if rng is None:
        rng = np.random.default_rng(seed)
    pr = math.radians(prior_deg)
    while True:
        v = rng.normal(size=3)
        prior = v / np.linalg.norm(v) * rng.uniform(0.0, 1.0) ** (1.0 / 3.0)
        phi = prior + rng.uniform(-pr, pr, 3)
        t = rng.uniform(0.0, box, 3)
        R = rotvec_matrix(phi)
        w = np.stack([rng.uniform(0, points[0], 4096), rng.uniform(0, points[1], 4096),
                      rng.uniform(0, points[2], 4096)], axis=1)
        X = w @ R.T + t
        vis = (X[:, 2] > 1.0) & (np.abs(X[:, 0]) <= fov * X[:, 2]) & (np.abs(X[:, 1]) <= fov * X[:, 2])
        if vis.mean() >= 0.25:
            break
    n_in = int(round(n * inlier_frac))
    sig = math.radians(noise_deg)
    out = np.empty((5, n))
    got = 0
    while got < n_in:
        m = 4 * (n_in - got) + 16
        w = np.stack([rng.uniform(0, points[0], m), rng.uniform(0, points[1], m),
                      rng.uniform(0, points[2], m)], axis=1)
        X = w @ R.T + t
        ok = (X[:, 2] > 1.0) & (np.abs(X[:, 0]) <= fov * X[:, 2]) & (np.abs(X[:, 1]) <= fov * X[:, 2])
        w, X = w[ok][: n_in - got], X[ok][: n_in - got]
        a = np.arctan2(X[:, 0], X[:, 2]) + rng.normal(0, sig, len(w))
        b = np.arctan2(X[:, 1], X[:, 2]) + rng.normal(0, sig, len(w))
        sl = slice(got, got + len(w))
        out[0:3, sl] = w.T
        out[3, sl], out[4, sl] = np.tan(a), np.tan(b)
        got += len(w)
    m = n - n_in
    out[0, n_in:] = rng.uniform(0, points[0], m)
    out[1, n_in:] = rng.uniform(0, points[1], m)
    out[2, n_in:] = rng.uniform(0, points[2], m)
    out[3, n_in:] = rng.uniform(-fov, fov, m)
    out[4, n_in:] = rng.uniform(-fov, fov, m)
    perm = rng.permutation(n)
    out = out[:, perm]
    inliers = np.nonzero(perm < n_in)[0]
    lo = np.concatenate([prior - pr, [0.0, 0.0, 0.0]])
    hi = np.concatenate([prior + pr, [box, box, box]])
    bounds = np.stack([lo, hi], axis=1).reshape(-1)
    eps = (hi - lo) / 2.0 ** levels
    truth = np.concatenate([phi, [t[2], t[0], t[1]]])
    return Problem(POSE6DOF, eps, bounds, np.ascontiguousarray(out), truth, inliers, "pose6dof",
                   dict(inlier_frac=inlier_frac, prior=prior, prior_deg=prior_deg, levels=levels))


def pose7dof(n: int = 5000, inlier_frac: float = 0.05, prior_deg: float = 30.0, box: float = 10.0,
             levels: int = 7, noise_deg: float = 0.1, points=(20.0, 20.0, 5.0), fov: float = 1.0,
             focal=(0.8, 1.2), focal_range=(0.6, 1.3), seed: int = SEED_BASE + 9,
             rng: np.random.Generator | None = None) -> Problem:
    """Camera posing with unknown focal length (7DoF, Sec. 4.2.2).  As the
    calibrated camera (points, prior, rotation, camera-frame translation
    (x, y, z) ~ U[0, box]^3, inliers and outliers), with a focal length
    f ~ U[focal]: inliers are seen at f (tan a, tan b), outliers at f times a
    random image point of the field of view.  Voting domain phi_prior +- prior per
    axis, z in [0, box], f in focal_range times the true f (the paper bounds f
    within [0.6, 1.3] of the ground truth), (x, y) in [0, box]^2; every coordinate
    splits ``levels`` times, and the tolerance of x and y is their leaf width."""
    if rng is None:
        rng = np.random.default_rng(seed)
    p6 = pose6dof(n=n, inlier_frac=inlier_frac, prior_deg=prior_deg, box=box, levels=levels,
                  noise_deg=noise_deg, points=points, fov=fov, rng=rng)
    f = rng.uniform(*focal)
    out = p6.params.copy()
    out[3:5] *= f
    lo6, hi6 = p6.bounds[0::2], p6.bounds[1::2]
    lo = np.concatenate([lo6[:4], [focal_range[0] * f], lo6[4:]])
    hi = np.concatenate([hi6[:4], [focal_range[1] * f], hi6[4:]])
    bounds = np.stack([lo, hi], axis=1).reshape(-1)
    eps = (hi - lo) / 2.0 ** levels
    truth = np.concatenate([p6.truth[:4], [f], p6.truth[4:]])
    meta = dict(p6.meta, focal=f)
    return Problem(POSE7DOF, eps, bounds, np.ascontiguousarray(out), truth, p6.inliers, "pose7dof", meta)


def radial5dof(n: int = 5000, inlier_frac: float = 0.05, prior_deg: float = 30.0, box: float = 10.0,
               levels: int = 7, noise_deg: float = 0.1, points=(20.0, 20.0, 5.0), fov: float = 1.0,
               xi_min: float = 0.2, focal=(0.8, 1.2), seed: int = SEED_BASE + 8,
               rng: np.random.Generator | None = None) -> Problem:
    """Radial-camera posing with unknown focal length (5DoF, Sec. 4.2.4).  World
    points uniform in [0, points_0] x [0, points_1] x [0, points_2]; camera frame
    X = R(phi) w + (-y, x, z), the radial camera's rows being (r1, -y) and (r2, x)
    (z and the focal length f ~ U[focal] are what the radial model leaves out).
    Truth: phi as for the calibrated camera (prior uniform in the unit ball, the
    rotation within +- prior per axis of it), -y, x, z ~ U[0, box] (redrawn until a
    quarter of the points are visible).  Inliers: points with X_3 > 1 m inside the
    field of view |X_1|, |X_2| <= fov X_3 and |X_1| >= xi_min X_3 (the surface
    divides by xi), seen at f (tan a, tan b) with a, b the bearing angles perturbed
    by N(0, noise); outliers: a random point with a random image point of the field
    of view, |xi| >= xi_min f.  Voting domain phi_prior +- prior per axis,
    y in [-box, 0], x in [0, box]; every coordinate splits ``levels`` times, and the
    tolerance of x is its leaf width (a constant distance)."""
    if rng is None:
        rng = np.random.default_rng(seed)
    pr = math.radians(prior_deg)

    def visible(X):
        return ((X[:, 2] > 1.0) & (np.abs(X[:, 0]) <= fov * X[:, 2]) & (np.abs(X[:, 1]) <= fov * X[:, 2])
                & (np.abs(X[:, 0]) >= xi_min * X[:, 2]))

    def world(m):
        return np.stack([rng.uniform(0, points[0], m), rng.uniform(0, points[1], m),
                         rng.uniform(0, points[2], m)], axis=1)

    while True:
        v = rng.normal(size=3)
        prior = v / np.linalg.norm(v) * rng.uniform(0.0, 1.0) ** (1.0 / 3.0)
        phi = prior + rng.uniform(-pr, pr, 3)
        t = rng.uniform(0.0, box, 3)                    # (-y, x, z)
        R = rotvec_matrix(phi)
        if visible(world(4096) @ R.T + t).mean() >= 0.25:
            break
    f = rng.uniform(*focal)
    n_in = int(round(n * inlier_frac))
    sig = math.radians(noise_deg)
    out = np.empty((5, n))
    got = 0
    while got < n_in:
        w = world(8 * (n_in - got) + 16)
        X = w @ R.T + t
        ok = visible(X)
        w, X = w[ok][: n_in - got], X[ok][: n_in - got]
        a = np.arctan2(X[:, 0], X[:, 2]) + rng.normal(0, sig, len(w))
        b = np.arctan2(X[:, 1], X[:, 2]) + rng.normal(0, sig, len(w))
        sl = slice(got, got + len(w))
        out[0:3, sl] = w.T
        out[3, sl], out[4, sl] = f * np.tan(a), f * np.tan(b)
        got += len(w)
    m = n - n_in
    out[0:3, n_in:] = world(m).T
    out[3, n_in:] = f * rng.choice([-1.0, 1.0], m) * rng.uniform(xi_min, fov, m)
    out[4, n_in:] = f * rng.uniform(-fov, fov, m)
    perm = rng.permutation(n)
    out = out[:, perm]
    inliers = np.nonzero(perm < n_in)[0]
    lo = np.concatenate([prior - pr, [-box, 0.0]])
    hi = np.concatenate([prior + pr, [0.0, box]])
    bounds = np.stack([lo, hi], axis=1).reshape(-1)
    eps = (hi - lo) / 2.0 ** levels
    truth = np.concatenate([phi, [-t[0], t[1]]])
    return Problem(RADIAL5DOF, eps, bounds, np.ascontiguousarray(out), truth, inliers, "radial5dof",
                   dict(inlier_frac=inlier_frac, prior=prior, prior_deg=prior_deg, levels=levels, focal=f))


def rays3d(n: int = 100_000, inlier_frac: float = 0.02, eps: float = 0.002, noise: float = 0.0005,
           slope: float = 2.0, seed: int = SEED_BASE + 5) -> Problem:
    """Rays y = a x + b, z = c x + d in the unit cube: ``inlier_frac`` of them pass
    within N(0, noise) (in y and z) of a common point p ~ U[0.2, 0.8]^3, the rest
    through a uniform point of the cube; slopes a, c ~ U[-slope, slope].  Voting
    domain [0, 1]^3 in (x, y, z); eps in every coordinate."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.2, 0.8, 3)
    n_in = int(round(n * inlier_frac))
    a = rng.uniform(-slope, slope, n)
    c = rng.uniform(-slope, slope, n)
    q = rng.uniform(0.0, 1.0, (n, 3))
    q[:n_in] = p
    b = q[:, 1] - a * q[:, 0]
    d = q[:, 2] - c * q[:, 0]
    b[:n_in] += rng.normal(0.0, noise, n_in)
    d[:n_in] += rng.normal(0.0, noise, n_in)
    out = np.stack([a, b, c, d])
    perm = rng.permutation(n)
    out = out[:, perm]
    inliers = np.nonzero(perm < n_in)[0]
    return Problem(RAYS3D, np.full(3, eps), np.array([0.0, 1.0, 0.0, 1.0, 0.0, 1.0]), np.ascontiguousarray(out),
                   p.copy(), inliers, "rays3d", dict(inlier_frac=inlier_frac))


def pointset2d(m: int = 200, outlier_frac: float = 0.0, eps: float = 0.01, noise: float = 0.002,
               seed: int = SEED_BASE + 6) -> Problem:
    """Two point sets of m points without known correspondences: A uniform in the
    annulus 0.25 <= |p| <= 1, B = s R A + t (+ N(0, noise)) with s ~ U[0.5, 1.5],
    rotation angle ~ U[-60, 60] deg, t ~ U[-1, 1]^2, and a fraction of B replaced by
    uniform points of [-2.5, 2.5]^2.  Every pair (p in A, q in B) is a surface
    (n = m^2); the m true pairs are the inliers.  Voting domain c, d in [-2, 2]
    (translation), a = s cos theta in [0.25, 1.75], b = s sin theta in [-1.5, 1.5]
    (the domain leaves out scale 0, where every pair with one q agrees); eps in
    every coordinate."""
    rng = np.random.default_rng(seed)
    r = np.sqrt(rng.uniform(0.25 ** 2, 1.0, m))
    ang = rng.uniform(0.0, 2 * math.pi, m)
    A = np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
    s, th = rng.uniform(0.5, 1.5), rng.uniform(-math.pi / 3, math.pi / 3)
    a, b = s * math.cos(th), s * math.sin(th)
    t = rng.uniform(-1.0, 1.0, 2)
    B = np.stack([a * A[:, 0] + b * A[:, 1] + t[0], -b * A[:, 0] + a * A[:, 1] + t[1]], axis=1)
    B += rng.normal(0.0, noise, B.shape)
    n_out = int(round(m * outlier_frac))
    out_idx = rng.choice(m, n_out, replace=False)
    B[out_idx] = rng.uniform(-2.5, 2.5, (n_out, 2))
    P = np.repeat(A, m, axis=0)
    Q = np.tile(B, (m, 1))
    params = np.stack([P[:, 0], P[:, 1], Q[:, 0], Q[:, 1]])
    truth_pairs = np.arange(m) * m + np.arange(m)
    keep = np.ones(m, bool)
    keep[out_idx] = False
    return Problem(POINTSET2D, np.full(4, eps), np.array([-2.0, 2.0, -2.0, 2.0, 0.25, 1.75, -1.5, 1.5]),
                   np.ascontiguousarray(params), np.array([t[0], t[1], a, b]), truth_pairs[keep], "pointset2d",
                   dict(m=m, scale=s, theta=th))


def affine4d(n: int = 10_000, inlier_frac: float = 0.05, eps: float = 0.02, noise: float = 0.002,
             seed: int = SEED_BASE + 7) -> Problem:
    """Points of R^4: (x1, x2, x3) uniform in [0, 1]^3; ``inlier_frac`` of them on a
    hyperplane x4 = a . (x1, x2, x3) + b (a ~ U[-1, 1]^3, b ~ U[0, 1]) plus
    N(0, noise) in x4, the rest with x4 ~ U[-1, 2] (a spread wider than a band of
    width 2 eps holds by chance).  Voting domain a in [-1, 1]^3, b in [-4, 5]; eps
    in every coordinate."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, 3)
    b = rng.uniform(0.0, 1.0)
    n_in = int(round(n * inlier_frac))
    x = rng.uniform(0.0, 1.0, (n, 3))
    x4 = rng.uniform(-1.0, 2.0, n)
    x4[:n_in] = x[:n_in] @ a + b + rng.normal(0.0, noise, n_in)
    out = np.concatenate([x.T, x4[None]], axis=0)
    perm = rng.permutation(n)
    out = out[:, perm]
    inliers = np.nonzero(perm < n_in)[0]
    return Problem(AFFINE4D, np.full(4, eps), np.array([-1.0, 1.0, -1.0, 1.0, -1.0, 1.0, -4.0, 5.0]),
                   np.ascontiguousarray(out), np.concatenate([a, [b]]), inliers, "affine4d",
                   dict(inlier_frac=inlier_frac))


# ---------------------------------------------------------------------------
# Standard workloads
# ---------------------------------------------------------------------------

WORKLOADS = {
    "line2d_n1e4": lambda: line2d(),
    "plane3d_n1e6": lambda: plane3d(),
    "pose3dof_n1e6": lambda: pose3dof(),
}


def random_small(family: int, n: int, seed: int, inlier_frac: float = 0.3, **kw) -> Problem:
    """Small instances for parity and invariance tests."""
    if family == LINE2D:
        return line2d(n=n, inlier_frac=inlier_frac, seed=seed, **kw)
    if family == PLANE3D_SPH:
        return plane3d(n=n, inlier_frac=inlier_frac, seed=seed, **kw)
    if family == POSE3DOF:
        return pose3dof(n=n, inlier_frac=inlier_frac, seed=seed, **kw)
    if family == POSE6DOF:
        return pose6dof(n=n, inlier_frac=inlier_frac, seed=seed, **kw)
    if family == RAYS3D:
        return rays3d(n=n, inlier_frac=inlier_frac, seed=seed, **kw)
    if family == POINTSET2D:
        return pointset2d(m=max(1, int(round(math.sqrt(n)))), seed=seed, **kw)
    if family == AFFINE4D:
        return affine4d(n=n, inlier_frac=inlier_frac, seed=seed, **kw)
    raise ValueError(family)
