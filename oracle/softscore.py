"""Oracle of the soft inlier score (test infrastructure only).

Plain PyTorch CPU FP64, the definition written out:
    S(p) = sum_i w_i exp(-u_i^2 / 2),  u_i^2 = sum_j (r_ij / tol_j)^2,
with r_ij the vertical residual of surface i at p in dependent coordinate j
(Eq. 1 of the paper in global form: r = p_dep - F(p_free; t) - g).  Gradients come
from torch.autograd on these CPU tensors.
Pins: tests/test_softscore_oracle.py (hand-computed single-surface values, exact
inliers, central finite differences, the plane double cover).
"""
from __future__ import annotations

import torch

LINE2D, PLANE3D_SPH, POSE3DOF, POSE6DOF, RAYS3D, POINTSET2D, AFFINE4D, RADIAL5DOF, POSE7DOF = range(1, 10)


def rotation(phi: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of the axis-angle vector phi (Rodrigues' formula)."""
    th2 = (phi * phi).sum()
    K = torch.stack([torch.stack([phi.new_zeros(()), -phi[2], phi[1]]),
                     torch.stack([phi[2], phi.new_zeros(()), -phi[0]]),
                     torch.stack([-phi[1], phi[0], phi.new_zeros(())])])
    if float(th2.detach()) < 1e-8:
        a = 1.0 - th2 / 6.0
        b = 0.5 - th2 / 24.0
    else:
        th = torch.sqrt(th2)
        a = torch.sin(th) / th
        b = (1.0 - torch.cos(th)) / th2
    return torch.eye(3, dtype=phi.dtype) + a * K + b * (K @ K)


def residuals(family: int, params: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    """[n, d-k] residuals (CPU float64)."""
    if family == LINE2D:                       # b = y - x m
        x, y = params[0], params[1]
        return (p[1] - (y - x * p[0]))[:, None]
    if family == PLANE3D_SPH:                  # d = q . (sin th cos ph, sin th sin ph, cos th)
        qx, qy, qz = params[0], params[1], params[2]
        nx = torch.sin(p[0]) * torch.cos(p[1])
        ny = torch.sin(p[0]) * torch.sin(p[1])
        nz = torch.cos(p[0])
        return (p[2] - (qx * nx + qy * ny + qz * nz))[:, None]
    if family == POSE3DOF:                     # x = w1 - (a cos - b sin), y = w2 - (a sin + b cos)
        w1, w2, a, b = params[0], params[1], params[2], params[3]
        c, s = torch.cos(p[0]), torch.sin(p[0])
        rx = p[1] - (w1 - (a * c - b * s))
        ry = p[2] - (w2 - (a * s + b * c))
        return torch.stack([rx, ry], dim=1)
    if family == AFFINE4D:                     # b = x4 - a . (x1, x2, x3)
        return (p[3] - (params[3] - (p[0] * params[0] + p[1] * params[1] + p[2] * params[2])))[:, None]
    if family == POINTSET2D:                   # (a, b) solving q = [[a, b], [-b, a]] p + (c, d)
        px, py, qx, qy = params[0], params[1], params[2], params[3]
        n2 = px * px + py * py
        ex, ey = qx - p[0], qy - p[1]
        return torch.stack([p[2] - (px * ex + py * ey) / n2, p[3] - (py * ex - px * ey) / n2], dim=1)
    if family == RAYS3D:                       # y = a x + b, z = c x + d
        a, b, c, d = params[0], params[1], params[2], params[3]
        return torch.stack([p[1] - (a * p[0] + b), p[2] - (c * p[0] + d)], dim=1)
    if family == POSE6DOF:                     # x = xi (r3 . w + z) - r1 . w, y = eta (r3 . w + z) - r2 . w
        X = rotation(p[0:3]) @ params[0:3]     # [3, n]
        depth = X[2] + p[3]
        rx = p[4] - (params[3] * depth - X[0])
        ry = p[5] - (params[4] * depth - X[1])
        return torch.stack([rx, ry], dim=1)
    if family == POSE7DOF:                     # x = xi (r3 . w + z) / f - r1 . w (and y with eta)
        X = rotation(p[0:3]) @ params[0:3]
        depth = (X[2] + p[3]) / p[4]
        rx = p[5] - (params[3] * depth - X[0])
        ry = p[6] - (params[4] * depth - X[1])
        return torch.stack([rx, ry], dim=1)
    if family == RADIAL5DOF:                   # x = eta (r1 . w - y) / xi - r2 . w
        X = rotation(p[0:3]) @ params[0:3]
        return (p[4] - (params[4] * (X[0] - p[3]) / params[3] - X[1]))[:, None]
    raise ValueError(family)


def softscore(family: int, params: torch.Tensor, p: torch.Tensor, weights: torch.Tensor, tol) -> torch.Tensor:
    r = residuals(family, params, p)
    tol = torch.as_tensor(tol, dtype=torch.float64)
    u2 = ((r / tol) ** 2).sum(dim=1)
    return (weights * torch.exp(-0.5 * u2)).sum()
