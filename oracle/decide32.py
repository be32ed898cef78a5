"""The float32 decisions that choose which samples exist (oracle, numpy float32).

Test infrastructure: only tests, smoke() and the bench's CPU-baseline leg use it.

Three integer outcomes of the renderer are decided by floating point: whether
a ray meets the performer's bounding box (Sec. 4.4 samples inside it), which
occupancy cell a sample falls in, and which cells of the posed occupancy
bitfield are set (empty-space skipping, Sec. 2.3).  Both sides take these
decisions in float32 with one fixed order of correctly rounded operations and
no fused multiply-add, so that they agree bit for bit.  Every expression below
states its evaluation order with parentheses; numpy float32 arithmetic rounds
after each operation.

Ray of pixel (u, v), camera world->camera (R, t) (OpenCV convention):
    o_k = -(((R0k t0) + (R1k t1)) + (R2k t2))
    a = ((u + 0.5) - cx) / fx,  b = ((v + 0.5) - cy) / fy
    w_k = ((R0k a) + (R1k b)) + R2k
    n = sqrt(((w0 w0) + (w1 w1)) + (w2 w2)),  d_k = w_k / n
Slab clip against [box_min, box_max] starting from [t_near, t_far]; an axis
with d_k == 0 misses when o_k is outside its slab and is skipped otherwise:
    ta = (bmin_k - o_k) / d_k, tb = (bmax_k - o_k) / d_k,
    lo = max(lo, min(ta, tb)), hi = min(hi, max(ta, tb)); hit iff lo < hi.
Midpoint samples: D = (hi - lo) / S, t_i = lo + ((i + 0.5) D), x_k = o_k + (t_i d_k).
Occupancy cell: h_k = (bmax_k - bmin_k) / G, c_k = clamp(floor((x_k - bmin_k) / h_k), 0, G-1),
linear index (c_z G + c_y) G + c_x, word index >> 5, bit index & 31.
Posed bitfield: cell centre y_k = bmin_k + ((j_k + 0.5) h_k); the cell is set iff for some
bone i the canonical point q = G_i y (q_r = (((R_r0 y0) + (R_r1 y1)) + (R_r2 y2)) + t_r)
lies in ellipsoid i dilated by half a cell diagonal dil = 0.5 sqrt(((h0 h0) + (h1 h1)) + (h2 h2)):
    v = q - centre, l_m = ((Q_m0 v0) + (Q_m1 v1)) + (Q_m2 v2), s_m = l_m / (r_m + dil),
    set iff ((s0 s0) + (s1 s1)) + (s2 s2) <= 1.
"""
from __future__ import annotations

import numpy as np

f32 = np.float32


def ray_dirs32(cam, px: np.ndarray, py: np.ndarray):
    """Ray origin o [3] and unit directions d [N][3] (float32) for pixels (px, py)."""
    R = np.asarray(cam.R, f32)
    t = np.asarray(cam.t, f32)
    o = np.empty(3, f32)
    for k in range(3):
        o[k] = -((R[0, k] * t[0] + R[1, k] * t[1]) + R[2, k] * t[2])
    a = ((px.astype(f32) + f32(0.5)) - f32(cam.cx)) / f32(cam.fx)
    b = ((py.astype(f32) + f32(0.5)) - f32(cam.cy)) / f32(cam.fy)
    w = np.stack([(R[0, k] * a + R[1, k] * b) + R[2, k] for k in range(3)], 1).astype(f32)
    n = np.sqrt((w[:, 0] * w[:, 0] + w[:, 1] * w[:, 1]) + w[:, 2] * w[:, 2])
    d = (w / n[:, None]).astype(f32)
    return o, d


def clip32(o: np.ndarray, d: np.ndarray, t_near, t_far, box_min, box_max):
    """Slab clip in float32: (lo [N], hi [N], hit [N] bool). o is [3] or [N][3]."""
    N = d.shape[0]
    o = np.broadcast_to(np.asarray(o, f32), (N, 3))
    lo = np.full(N, f32(t_near), f32)
    hi = np.full(N, f32(t_far), f32)
    miss = np.zeros(N, bool)
    bmin = np.asarray(box_min, f32)
    bmax = np.asarray(box_max, f32)
    with np.errstate(divide="ignore", invalid="ignore"):
        for k in range(3):
            dk, ok = d[:, k], o[:, k]
            zero = dk == 0
            miss |= zero & ((ok < bmin[k]) | (ok > bmax[k]))
            ta = (bmin[k] - ok) / dk
            tb = (bmax[k] - ok) / dk
            lo = np.where(zero, lo, np.maximum(lo, np.minimum(ta, tb))).astype(f32)
            hi = np.where(zero, hi, np.minimum(hi, np.maximum(ta, tb))).astype(f32)
    hit = (~miss) & (lo < hi)
    return lo, hi, hit


def sample_points32(o, d, lo, hi, n_samples: int):
    """Midpoint samples x [N][S][3] (float32) for rays already clipped to [lo, hi]."""
    N = d.shape[0]
    o = np.broadcast_to(np.asarray(o, f32), (N, 3))
    D = (hi - lo) / f32(n_samples)
    s = np.arange(n_samples, dtype=f32) + f32(0.5)
    t = lo[:, None] + (s[None, :] * D[:, None])
    return (o[:, None, :] + (t[:, :, None] * d[:, None, :])).astype(f32)


def cell_of32(x: np.ndarray, box_min, box_max, grid: int) -> np.ndarray:
    """Linear occupancy-cell index of float32 points x [..., 3]."""
    bmin = np.asarray(box_min, f32)
    h = ((np.asarray(box_max, f32) - bmin) / f32(grid)).astype(f32)
    c = np.floor((x - bmin) / h).astype(np.int64)
    c = np.clip(c, 0, grid - 1)
    return (c[..., 2] * grid + c[..., 1]) * grid + c[..., 0]


def bit_test(bits: np.ndarray, cell: np.ndarray) -> np.ndarray:
    return ((bits[cell >> 5] >> (cell & 31).astype(np.uint32)) & 1).astype(bool)


def posed_bitfield32(G: np.ndarray, ellipsoids: np.ndarray, box_min, box_max, grid: int = 128) -> np.ndarray:
    """Posed occupancy bitfield [grid^3 / 32] uint32 from float32 G [K][12] and ellipsoids [K][15]."""
    bmin = np.asarray(box_min, f32)
    h = ((np.asarray(box_max, f32) - bmin) / f32(grid)).astype(f32)
    dil = f32(0.5) * np.sqrt((h[0] * h[0] + h[1] * h[1]) + h[2] * h[2])
    j = np.arange(grid, dtype=f32) + f32(0.5)
    cz, cy, cx = np.meshgrid(bmin[2] + j * h[2], bmin[1] + j * h[1], bmin[0] + j * h[0], indexing="ij")
    y = [cx.ravel().astype(f32), cy.ravel().astype(f32), cz.ravel().astype(f32)]
    occ = np.zeros(grid ** 3, bool)
    G = np.asarray(G, f32).reshape(-1, 3, 4)
    E = np.asarray(ellipsoids, f32)
    for i in range(G.shape[0]):
        R = G[i]
        q = [((R[r, 0] * y[0] + R[r, 1] * y[1]) + R[r, 2] * y[2]) + R[r, 3] for r in range(3)]
        v = [q[k] - E[i, k] for k in range(3)]
        Q = E[i, 3:12].reshape(3, 3)
        rad = E[i, 12:15]
        s = [(((Q[m, 0] * v[0] + Q[m, 1] * v[1]) + Q[m, 2] * v[2]) / (rad[m] + dil)) for m in range(3)]
        occ |= ((s[0] * s[0] + s[1] * s[1]) + s[2] * s[2]) <= f32(1.0)
    bits = np.zeros(grid ** 3 // 32, np.uint32)
    idx = np.nonzero(occ)[0]
    np.bitwise_or.at(bits, idx >> 5, (np.uint32(1) << (idx & 31).astype(np.uint32)))
    return bits
