"""Forward kinematics -> per-bone observation-to-canonical transforms (oracle, FP64).

Test infrastructure: only tests, smoke() and the bench's CPU-baseline leg use it.

Sec. 4.2 defines the skeleton motion basis G_i(x) = R_i x + t_i, "calculated
from the corresponding body pose theta^o".  A pose theta = (J, Omega) is the
joints plus one joint angle per joint (Sec. 4.1); the canonical pose is the
rest pose.  With B_i the rigid map that carries bone i's canonical body part
to its observed place, G_i = B_i^{-1}:

    A_root = [Rot(omega_0) | J_0 + root_t]
    A_i    = A_parent(i) o [Rot(omega_i) | J_i - J_parent(i)]
    B_i(x) = A_i.R (x - J_i) + A_i.t
    G_i(x) = A_i.R^T (x - A_i.t) + J_i       i.e. R_i = A_i.R^T, t_i = J_i - A_i.R^T A_i.t

Rot(omega) is the axis-angle rotation (Rodrigues' formula).
"""
from __future__ import annotations

import numpy as np


def rodrigues(aa: np.ndarray) -> np.ndarray:
    """Axis-angle [..., 3] -> rotation matrix [..., 3, 3] (FP64)."""
    aa = np.asarray(aa, np.float64)
    th = np.linalg.norm(aa, axis=-1)
    out = np.empty(aa.shape[:-1] + (3, 3))
    flat_aa = aa.reshape(-1, 3)
    flat_th = th.reshape(-1)
    flat_out = out.reshape(-1, 3, 3)
    for n in range(flat_aa.shape[0]):
        a, t = flat_aa[n], flat_th[n]
        K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
        if t < 1e-12:
            flat_out[n] = np.eye(3) + K
        else:
            K = K / t
            flat_out[n] = np.eye(3) + np.sin(t) * K + (1.0 - np.cos(t)) * (K @ K)
    return out


def posed_joints(parents, rest_joints, axis_angle, root_t):
    """World rotation and position of every joint in the observed pose: (A_R [K,3,3], A_t [K,3])."""
    J = np.asarray(rest_joints, np.float64)
    rot = rodrigues(axis_angle)
    K = J.shape[0]
    AR = np.zeros((K, 3, 3))
    At = np.zeros((K, 3))
    for i in range(K):
        p = parents[i]
        if p < 0:
            AR[i] = rot[i]
            At[i] = J[i] + np.asarray(root_t, np.float64)
        else:
            AR[i] = AR[p] @ rot[i]
            At[i] = AR[p] @ (J[i] - J[p]) + At[p]
    return AR, At


def bone_transforms(parents, rest_joints, axis_angle, root_t):
    """G_i = (R_i [K,3,3], t_i [K,3]) in FP64, mapping observation -> canonical."""
    AR, At = posed_joints(parents, rest_joints, axis_angle, root_t)
    J = np.asarray(rest_joints, np.float64)
    R = np.transpose(AR, (0, 2, 1))
    t = J - np.einsum("kij,kj->ki", R, At)
    return R, t


def bone_transforms_f32(parents, rest_joints, axis_angle, root_t) -> np.ndarray:
    """The FP64 transforms rounded to float32, packed [K][12] as rows [R | t]."""
    R, t = bone_transforms(parents, rest_joints, axis_angle, root_t)
    G = np.concatenate([R, t[:, :, None]], axis=2)         # [K][3][4]
    return G.reshape(-1, 12).astype(np.float32)
