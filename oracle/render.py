"""Rays, sampling, compositing and loss (oracle, FP64, plain PyTorch CPU ops).

Test infrastructure: only tests, smoke() and the bench's CPU-baseline leg use it.

Volume rendering follows Sec. 2.1: the quadrature of Eq. 3 read as
    C^ = sum_i T_i (1 - exp(-sigma_i delta_i)) c_i,   T_i = prod_{j<i} (1 - alpha_j)
(the typeset parenthesis of Eq. 3 closes after c_i; the vanilla-NeRF form is
used), with the likelihood augmentation of Sec. 4.4:
    alpha_i = (1 - exp(-sigma_i delta_i)) * min(S_i, 1)
where S_i is the denominator of Eq. lbs at the sample.  The pixel is
(C^ + T_final bg, 1 - T_final).  No early termination: the oracle composites
every sample.  Samples lie inside the performer's bounding box (Sec. 4.4):
each ray is clipped to the box and split into S equal bins; rendering uses
bin midpoints with delta_i = (hi - lo) / S, training draws a stratified point
per bin, delta_i = t_{i+1} - t_i and delta_{S-1} = hi - t_{S-1}.  A sample the
occupancy bitfield marks empty has sigma = 0 (empty-space skipping, Sec. 2.3).
The loss is the mean over rays and channels of the squared error (Sec. 2.1,
Sec. 5.2; the LPIPS term needs pretrained weights and is not part of it).
"""
from __future__ import annotations

import numpy as np
import torch

from . import decide32, fk, refine, rng
from .field import F64, Params, field, t64


def rays64(cam, px: np.ndarray, py: np.ndarray):
    """FP64 ray origin [3] and unit directions [N][3] of pixels (px, py) (OpenCV camera)."""
    R = t64(np.asarray(cam.R, np.float32))
    t = t64(np.asarray(cam.t, np.float32))
    o = -(R.T @ t)
    a = (t64(px) + 0.5 - cam.cx) / cam.fx
    b = (t64(py) + 0.5 - cam.cy) / cam.fy
    dirc = torch.stack([a, b, torch.ones_like(a)], 1)
    w = dirc @ R                        # R^T applied to each row vector
    return o, w / torch.linalg.norm(w, dim=1, keepdim=True)


def clip64(o, d, t_near, t_far, box_min, box_max):
    """FP64 slab clip: (lo [N], hi [N]); an empty interval has hi <= lo."""
    N = d.shape[0]
    o = o.expand(N, 3) if o.dim() == 1 else o
    lo = torch.full((N,), float(t_near), dtype=F64)
    hi = torch.full((N,), float(t_far), dtype=F64)
    bmin, bmax = t64(box_min), t64(box_max)
    for k in range(3):
        dk = d[:, k]
        zero = dk == 0
        safe = torch.where(zero, torch.ones_like(dk), dk)
        ta = (bmin[k] - o[:, k]) / safe
        tb = (bmax[k] - o[:, k]) / safe
        lo = torch.where(zero, lo, torch.maximum(lo, torch.minimum(ta, tb)))
        hi = torch.where(zero, hi, torch.minimum(hi, torch.maximum(ta, tb)))
    return lo, hi


def sample_t(lo, hi, n_samples: int, u=None):
    """Sample depths t [N][S] and spacings delta [N][S] inside [lo, hi]."""
    D = (hi - lo) / n_samples
    i = torch.arange(n_samples, dtype=F64)[None, :]
    if u is None:
        t = lo[:, None] + (i + 0.5) * D[:, None]
        delta = D[:, None].expand(-1, n_samples).clone()
    else:
        t = lo[:, None] + (i + t64(u)) * D[:, None]
        delta = torch.cat([t[:, 1:] - t[:, :-1], (hi[:, None] - t[:, -1:])], 1)
    return t, delta


def composite(rgb, alpha, bg):
    """Front-to-back compositing of rgb [N][S][3], alpha [N][S] -> (rgba [N][4], weights [N][S])."""
    one_minus = 1.0 - alpha
    T = torch.cumprod(torch.cat([torch.ones_like(alpha[:, :1]), one_minus], 1), 1)
    Ti, Tf = T[:, :-1], T[:, -1]
    w = Ti * alpha
    C = (w[:, :, None] * rgb).sum(1) + Tf[:, None] * t64(bg)[None, :]
    return torch.cat([C, (1.0 - Tf)[:, None]], 1), w


def sample_alpha(out, delta, live):
    """alpha_i = (1 - exp(-sigma_i delta_i)) * min(S_i, 1), zero outside the box or where skipped."""
    a = (1.0 - torch.exp(-out["sigma"] * delta)) * torch.clamp(out["S"], max=1.0)
    keep = out["inside"] & live
    return torch.where(keep, a, torch.zeros((), dtype=F64))


def pose_inputs(subj: dict, axis_angle, root_t, refiner=None):
    """FP64 G (R [K,3,3], t [K,3]) and the flattened joint angles Omega [3K] that condition
    MLP_res; with `refiner` (MLP_theta layers, Sec. 4.1) both are those of the refined pose."""
    omega = t64(np.asarray(axis_angle, np.float32)).reshape(-1)
    if refiner is not None:
        return refine.refined_pose(subj["parents"], subj["rest_joints"], axis_angle, root_t, refiner)
    R, t = fk.bone_transforms(subj["parents"], subj["rest_joints"], axis_angle, root_t)
    return torch.from_numpy(R), torch.from_numpy(t), omega


def render_pixels(subj: dict, P: Params, pose, cam, px, py, use_occupancy: bool,
                  grid: int = 128, chunk: int = 1024, alpha=None, return_counts: bool = False,
                  bits=None, refiner=None):
    """RGBA [N][4] (float64) of pixels (px, py) for one pose and camera.

    The box-hit and occupancy decisions come from `decide32` (float32, the
    kernel's precision); everything else is FP64.  `bits` (uint32 words of a
    grid^3 posed bitfield) replaces the ellipsoid bitfield when given.
    """
    axis_angle, root_t = pose
    G_R, G_t, omega = pose_inputs(subj, axis_angle, root_t, refiner)
    px = np.asarray(px)
    py = np.asarray(py)
    o32, d32 = decide32.ray_dirs32(cam, px, py)
    lo32, hi32, hit32 = decide32.clip32(o32, d32, cam.t_near, cam.t_far, subj["box_min"], subj["box_max"])
    S = cam.n_samples
    if use_occupancy:
        if bits is None:
            G32 = fk.bone_transforms_f32(subj["parents"], subj["rest_joints"], axis_angle, root_t)
            bits = decide32.posed_bitfield32(G32, subj["ellipsoids"], subj["box_min"], subj["box_max"], grid)
        x32 = decide32.sample_points32(o32, d32, lo32, hi32, S)
        live = decide32.bit_test(bits, decide32.cell_of32(x32, subj["box_min"], subj["box_max"], grid))
        live &= hit32[:, None]
    else:
        live = np.broadcast_to(hit32[:, None], (px.shape[0], S)).copy()
    o, d = rays64(cam, px, py)
    lo, hi = clip64(o, d, cam.t_near, cam.t_far, subj["box_min"], subj["box_max"])
    hit = torch.from_numpy(hit32) & (hi > lo)
    bg = t64(np.asarray(cam.bg, np.float32))
    out = torch.zeros(px.shape[0], 4, dtype=F64)
    out[:, :3] = bg
    live_t = torch.from_numpy(np.ascontiguousarray(live))
    for c0 in range(0, px.shape[0], chunk):
        sl = slice(c0, c0 + chunk)
        h = hit[sl]
        if not bool(h.any()):
            continue
        idx = torch.nonzero(h).squeeze(1) + c0
        t, delta = sample_t(lo[idx], hi[idx], S)
        x = o[None, None, :] + t[:, :, None] * d[idx][:, None, :]
        f = field(x.reshape(-1, 3), P, G_R, G_t, omega, alpha)
        a = sample_alpha(f, delta.reshape(-1), live_t[idx].reshape(-1)).reshape(-1, S)
        rgba, _ = composite(f["rgb"].reshape(-1, S, 3), a, bg)
        out[idx] = rgba
    if return_counts:
        return out, live.sum(1)
    return out


def render_image(subj: dict, pose, cam, use_occupancy: bool, **kw) -> torch.Tensor:
    """Full image [H][W][4] (float64)."""
    P = Params(subj)
    py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    out = render_pixels(subj, P, pose, cam, px.ravel(), py.ravel(), use_occupancy, **kw)
    return out.reshape(cam.height, cam.width, 4)


def train_loss(subj: dict, P: Params, frames: dict, batch: dict, target_rgb, step_seed: int,
               n_samples: int, bg, alpha=None, ray_offset: int = 0, loss_weight: float = 1.0,
               refiner=None):
    """loss_weight x mean squared error over rays and channels of one training batch (no
    occupancy, no ERT); Sec. 5.2 weights the MSE term by lambda_mse = 0.2.  `refiner`
    (MLP_theta layers) corrects each frame's pose (Sec. 4.1).

    frames: axis_angle [F][24][3], root_t [F][3], cameras [F]; batch: frame, px, py [N].
    """
    fr = np.asarray(batch["frame"])
    px = np.asarray(batch["px"])
    py = np.asarray(batch["py"])
    N = fr.shape[0]
    u_all = rng.jitter(step_seed, N, n_samples, ray_offset)
    tgt = t64(np.asarray(target_rgb, np.float32))
    bgt = t64(np.asarray(bg, np.float32))
    pred = torch.zeros(N, 3, dtype=F64) + bgt
    pred_list = []
    for f in np.unique(fr):
        sel = np.nonzero(fr == f)[0]
        cam = frames["cameras"][f]
        G_R, G_t, omega = pose_inputs(subj, frames["axis_angle"][f], frames["root_t"][f], refiner)
        o32, d32 = decide32.ray_dirs32(cam, px[sel], py[sel])
        _, _, hit32 = decide32.clip32(o32, d32, cam.t_near, cam.t_far, subj["box_min"], subj["box_max"])
        o, d = rays64(cam, px[sel], py[sel])
        lo, hi = clip64(o, d, cam.t_near, cam.t_far, subj["box_min"], subj["box_max"])
        h = torch.from_numpy(hit32) & (hi > lo)
        if not bool(h.any()):
            continue
        hs = torch.nonzero(h).squeeze(1)
        rows = sel[hs.numpy()]
        t, delta = sample_t(lo[hs], hi[hs], n_samples, u_all[rows])
        x = o[None, None, :] + t[:, :, None] * d[hs][:, None, :]
        out = field(x.reshape(-1, 3), P, G_R, G_t, omega, alpha)
        a = sample_alpha(out, delta.reshape(-1), torch.ones(x.shape[0] * n_samples, dtype=torch.bool))
        rgba, _ = composite(out["rgb"].reshape(-1, n_samples, 3), a.reshape(-1, n_samples), bgt)
        pred_list.append((torch.from_numpy(rows), rgba[:, :3]))
    for rows, rgb in pred_list:
        pred = pred.index_put((rows,), rgb)
    return loss_weight * ((pred - tgt) ** 2).mean(), pred
