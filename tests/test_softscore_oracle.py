"""Pins of the soft-score oracle (CPU)."""
import math

import numpy as np
import torch

from oracle import softscore as ss
from paper_2107_11810_gb300 import inputs


def test_single_line_hand_value():
    # point (x, y) = (0.5, 0.25); at (m, b) = (0.5, 0.1) the dual-line residual is
    # b - (y - x m) = 0.1 - 0 = 0.1; with tol 0.1, u = 1 and S = exp(-1/2)
    prm = torch.tensor([[0.5], [0.25]], dtype=torch.float64)
    p = torch.tensor([0.5, 0.1], dtype=torch.float64)
    s = ss.softscore(ss.LINE2D, prm, p, torch.ones(1, dtype=torch.float64), [0.1])
    assert abs(float(s) - math.exp(-0.5)) < 1e-15


def test_single_pose_hand_value():
    # camera at (10, 20), yaw 0.3; the surface of a point seen at (a, b) = (3, 4)
    # passes exactly through the camera position at that yaw: r = 0, S = 1;
    # moving x by tol gives u = 1
    yaw, cx, cy, a, b = 0.3, 10.0, 20.0, 3.0, 4.0
    w1 = cx + (a * math.cos(yaw) - b * math.sin(yaw))
    w2 = cy + (a * math.sin(yaw) + b * math.cos(yaw))
    prm = torch.tensor([[w1], [w2], [a], [b]], dtype=torch.float64)
    w = torch.ones(1, dtype=torch.float64)
    s0 = ss.softscore(ss.POSE3DOF, prm, torch.tensor([yaw, cx, cy], dtype=torch.float64), w, [0.25, 0.25])
    s1 = ss.softscore(ss.POSE3DOF, prm, torch.tensor([yaw, cx + 0.25, cy], dtype=torch.float64), w, [0.25, 0.25])
    assert abs(float(s0) - 1.0) < 1e-12
    assert abs(float(s1) - math.exp(-0.5)) < 1e-12


def test_exact_inliers_sum_of_weights_and_plane_double_cover():
    rng = np.random.default_rng(3)
    th, ph = 0.7, 2.1
    n = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    d = 0.3
    # points exactly on the plane n . q = d
    q = rng.uniform(-1, 1, size=(40, 3))
    q -= np.outer(q @ n - d, n)
    prm = torch.from_numpy(q.T.copy())
    w = torch.from_numpy(rng.integers(0, 2, 40).astype(np.float64))
    p = torch.tensor([th, ph, d], dtype=torch.float64)
    s = ss.softscore(ss.PLANE3D_SPH, prm, p, w, [0.01])
    assert abs(float(s) - float(w.sum())) < 1e-9
    # (theta, phi, d) and (pi - theta, phi + pi, -d) are the same plane
    q2 = rng.uniform(0, 1, size=(30, 3))
    prm2 = torch.from_numpy(q2.T.copy())
    w2 = torch.ones(30, dtype=torch.float64)
    a = ss.softscore(ss.PLANE3D_SPH, prm2, p, w2, [0.2])
    b = ss.softscore(ss.PLANE3D_SPH, prm2, torch.tensor([math.pi - th, ph + math.pi, -d], dtype=torch.float64), w2,
                     [0.2])
    assert abs(float(a) - float(b)) < 1e-12


def test_oracle_gradients_match_central_differences():
    for fam, mk, tol in [(ss.LINE2D, lambda: inputs.line2d(n=200, seed=4), [0.05]),
                         (ss.PLANE3D_SPH, lambda: inputs.plane3d(n=200, seed=5), [0.05]),
                         (ss.POSE3DOF, lambda: inputs.pose3dof(n=200, seed=6), [2.0, 2.0]),
                         (ss.POSE6DOF, lambda: inputs.pose6dof(n=200, seed=7), [0.5, 0.5]),
                         (ss.RAYS3D, lambda: inputs.rays3d(n=200, seed=9), [0.05, 0.05]),
                         (ss.POINTSET2D, lambda: inputs.pointset2d(m=15, seed=10), [0.05, 0.05]),
                         (ss.AFFINE4D, lambda: inputs.affine4d(n=200, seed=11), [0.05]),
                         (ss.RADIAL5DOF, lambda: inputs.radial5dof(n=200, seed=12), [0.5]),
                         (ss.POSE7DOF, lambda: inputs.pose7dof(n=200, seed=13), [0.5, 0.5])]:
        prob = mk()
        prm = torch.from_numpy(prob.params.copy()).requires_grad_(True)
        p = torch.tensor(prob.truth, dtype=torch.float64) + 0.003
        p.requires_grad_(True)
        w = torch.ones(prob.n, dtype=torch.float64)
        s = ss.softscore(fam, prm, p, w, tol)
        gp, gq = torch.autograd.grad(s, [p, prm])
        h = 1e-6
        for j in range(p.numel()):
            e = torch.zeros_like(p)
            e[j] = h
            with torch.no_grad():
                fd = (ss.softscore(fam, prm, p + e, w, tol) - ss.softscore(fam, prm, p - e, w, tol)) / (2 * h)
            assert abs(float(fd) - float(gp[j])) <= 1e-6 * max(1.0, abs(float(fd)))
        for (m, i) in [(0, 0), (prm.shape[0] - 1, 7)]:
            e = torch.zeros_like(prm)
            e[m, i] = h
            with torch.no_grad():
                fd = (ss.softscore(fam, prm + e, p, w, tol) - ss.softscore(fam, prm - e, p, w, tol)) / (2 * h)
            assert abs(float(fd) - float(gq[m, i])) <= 1e-6 * max(1.0, abs(float(fd)))


def test_pose6_residuals_equal_the_textbook_projection():
    # x - F_x = X_1 - xi X_3 with X = R w + t the point in the camera frame (scipy's
    # rotation, independent of the oracle's): zero for a noise-free match
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(8)
    phi, t = np.array([0.4, -0.7, 0.2]), np.array([2.0, 3.0, 6.0])
    R = Rotation.from_rotvec(phi).as_matrix()
    w = rng.uniform(0, 5, size=(20, 3))
    X = w @ R.T + t
    xi, eta = X[:, 0] / X[:, 2], X[:, 1] / X[:, 2]
    prm = torch.from_numpy(np.stack([w[:, 0], w[:, 1], w[:, 2], xi, eta]))
    p = torch.tensor([*phi, t[2], t[0], t[1]], dtype=torch.float64)
    r = ss.residuals(ss.POSE6DOF, prm, p)
    assert float(r.abs().max()) < 1e-12
    s = ss.softscore(ss.POSE6DOF, prm, p, torch.ones(20, dtype=torch.float64), [0.1, 0.1])
    assert abs(float(s) - 20.0) < 1e-9
    # a perturbed image point: the residual is the lateral offset X_3 (xi' - xi)
    prm2 = prm.clone()
    prm2[3] = prm2[3] + 0.01
    r2 = ss.residuals(ss.POSE6DOF, prm2, p)
    assert np.allclose(r2[:, 0].numpy(), -0.01 * X[:, 2], atol=1e-12)


def test_radial_and_focal_residuals_equal_the_textbook_projections():
    # radial camera rows (r1, -y), (r2, x): a noise-free match satisfies
    # eta X_1 = xi X_2 with X_1 = r1 . w - y, X_2 = r2 . w + x, and the residual of a
    # perturbed eta is the change of x; 7DoF: f (X_1, X_2) / X_3 = (xi, eta) with
    # X = R w + (x, y, z) (scipy's rotation, independent of the oracle's)
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(9)
    phi, t, f = np.array([0.3, -0.5, 0.6]), np.array([2.0, 3.0, 6.0]), 1.15
    R = Rotation.from_rotvec(phi).as_matrix()
    w = rng.uniform(0, 5, size=(20, 3))
    Rw = w @ R.T
    X = Rw + t
    xi, eta = f * X[:, 0] / X[:, 2], f * X[:, 1] / X[:, 2]
    prm = torch.from_numpy(np.stack([w[:, 0], w[:, 1], w[:, 2], xi, eta]))
    # radial: (phi, y, x) with X_1 = r1 . w - y, X_2 = r2 . w + x
    p5 = torch.tensor([*phi, -t[0], t[1]], dtype=torch.float64)
    assert float(ss.residuals(ss.RADIAL5DOF, prm, p5).abs().max()) < 1e-12
    prm2 = prm.clone()
    prm2[4] = prm2[4] + 0.01
    r2 = ss.residuals(ss.RADIAL5DOF, prm2, p5)[:, 0].numpy()
    assert np.allclose(r2, -0.01 * X[:, 0] / xi, atol=1e-12)
    # 7DoF: (phi, z, f, x, y)
    p7 = torch.tensor([*phi, t[2], f, t[0], t[1]], dtype=torch.float64)
    assert float(ss.residuals(ss.POSE7DOF, prm, p7).abs().max()) < 1e-12
    s7 = ss.softscore(ss.POSE7DOF, prm, p7, torch.ones(20, dtype=torch.float64), [0.1, 0.1])
    assert abs(float(s7) - 20.0) < 1e-9
