"""Pose refiner (Sec. 4.1) and the differentiable forward kinematics it feeds
(oracle, FP64, plain PyTorch CPU ops).

Test infrastructure: only tests, smoke() and the bench's CPU-baseline leg use it.

The estimated pose theta = (J, Omega) is corrected by a small MLP:

    Delta_Omega = MLP_theta(Omega)          (Sec. 4.1)
    theta^o     = (J, Delta_Omega (x) Omega)

Readings (the paper prints no sizes and no formula for the composition):
  * MLP_theta sees the joint angles of the K - 1 non-root joints (axis-angle,
    3 (K - 1) values) and returns one axis-angle correction per non-root joint;
    ReLU hidden layers, linear output.  The root keeps its estimated rotation
    and translation.
  * Delta_omega_j (x) omega_j is the composition of rotations
    Rot(Delta_omega_j) Rot(omega_j): the correction acts after the estimate in
    the parent's frame.
  * the joints J are kept; G_i follows from the refined local rotations by the
    forward kinematics of fk.py (A_i = A_parent o [Rot_i | J_i - J_parent],
    G_i = A_i^{-1} composed with the rest placement).
  * MLP_res is conditioned on the updated joint angles Omega^o (the residual
    network's figure caption): omega^o_j = Log(Rot(Delta_omega_j) Rot(omega_j)),
    the axis-angle of the composed rotation (rotations below pi), and
    omega^o_0 = omega_0.
"""
from __future__ import annotations

import numpy as np
import torch

from .field import F64, t64


def rodrigues_t(v: torch.Tensor) -> torch.Tensor:
    """Axis-angle [..., 3] -> rotation [..., 3, 3]: I + A K + B K^2 with K = [v]_x,
    A = sin(th) / th, B = (1 - cos(th)) / th^2, th = |v|; the Taylor forms of A and B
    below th^2 = 1e-12 keep the map (and its derivative) exact near zero."""
    th2 = (v * v).sum(-1)
    small = th2 < 1e-12
    th = torch.sqrt(torch.clamp(th2, min=1e-12))
    A = torch.where(small, 1.0 - th2 / 6.0, torch.sin(th) / th)
    B = torch.where(small, 0.5 - th2 / 24.0, (1.0 - torch.cos(th)) / (th * th))
    z = torch.zeros_like(v[..., 0])
    K = torch.stack([torch.stack([z, -v[..., 2], v[..., 1]], -1),
                     torch.stack([v[..., 2], z, -v[..., 0]], -1),
                     torch.stack([-v[..., 1], v[..., 0], z], -1)], -2)
    eye = torch.eye(3, dtype=v.dtype).expand(K.shape)
    return eye + A[..., None, None] * K + B[..., None, None] * (K @ K)


def rot_log_t(R: torch.Tensor) -> torch.Tensor:
    """Rotation [..., 3, 3] -> axis-angle [..., 3] with angle in [0, pi):
    a = (R_32 - R_23, R_13 - R_31, R_21 - R_12) / 2 = sin(th) n, cos(th) = (tr R - 1) / 2,
    v = th / sin(th) a, the ratio by its Taylor form 1 + th^2 / 6 where sin(th) < 1e-8."""
    a = 0.5 * torch.stack([R[..., 2, 1] - R[..., 1, 2], R[..., 0, 2] - R[..., 2, 0], R[..., 1, 0] - R[..., 0, 1]], -1)
    c = 0.5 * (R[..., 0, 0] + R[..., 1, 1] + R[..., 2, 2] - 1.0)
    s2 = (a * a).sum(-1)
    small = s2 < 1e-16
    s = torch.sqrt(torch.clamp(s2, min=1e-16))
    th = torch.atan2(s, c)
    k = torch.where(small, 1.0 + th * th / 6.0, th / s)
    return k[..., None] * a


def refiner_forward(layers, omega_nonroot: torch.Tensor) -> torch.Tensor:
    """MLP_theta: [3(K-1)] joint angles -> [3(K-1)] corrections (ReLU hidden layers)."""
    h = omega_nonroot
    for W, b in layers[:-1]:
        h = torch.relu(W @ h + b)
    W, b = layers[-1]
    return W @ h + b


def refined_transforms(parents, rest_joints, axis_angle, root_t, layers=None):
    """(G_R [K,3,3], G_t [K,3]) of the refined pose, FP64, differentiable in `layers`.

    layers None: no correction (the estimated pose)."""
    R, t, _ = refined_pose(parents, rest_joints, axis_angle, root_t, layers)
    return R, t


def refined_pose(parents, rest_joints, axis_angle, root_t, layers=None):
    """(G_R [K,3,3], G_t [K,3], Omega^o [3K]): the refined pose's transforms and updated
    joint angles, FP64, differentiable in `layers`."""
    J = t64(np.asarray(rest_joints, np.float64))
    om = t64(np.asarray(axis_angle, np.float32)).reshape(-1, 3)
    K = om.shape[0]
    rot = rodrigues_t(om)
    omega_o = om
    if layers is not None:
        delta = refiner_forward(layers, om[1:].reshape(-1)).reshape(-1, 3)
        rot = torch.cat([rot[:1], rodrigues_t(delta) @ rot[1:]], 0)
        omega_o = torch.cat([om[:1], rot_log_t(rot[1:])], 0)
    rt = t64(np.asarray(root_t if root_t is not None else np.zeros(3), np.float32))
    AR, At = [None] * K, [None] * K
    for i in range(K):
        p = int(parents[i])
        if p < 0:
            AR[i] = rot[i]
            At[i] = J[i] + rt
        else:
            AR[i] = AR[p] @ rot[i]
            At[i] = AR[p] @ (J[i] - J[p]) + At[p]
    R = torch.stack([a.T for a in AR])
    t = J - torch.einsum("kij,kj->ki", R, torch.stack(At))
    return R, t, omega_o.reshape(-1)
