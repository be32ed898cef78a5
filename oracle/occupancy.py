"""Occupancy grids from the field's own density (oracle, FP64, plain PyTorch CPU ops).

Test infrastructure: only tests, smoke() and the bench's CPU-baseline leg use it.

Empty-space skipping (Sec. 2.3) needs, for every pose, the cells of the box in
which the performer can have density.  Ellipsoids fixed by hand do not follow a
trained subject, so the set is taken from the canonical field itself and then
carried to the observed pose by the same warp that the samples go through:

  cell centres   y_c = bmin + (c + 1/2) h,  h = (bmax - bmin) / G, for c in 0..G-1
                 per axis; linear index (c_z G + c_y) G + c_x.
  canonical      marked(c) = sigma(y_c) > tau, sigma = softplus(o_3) of MLP_nerf
                 on the hash encoding of the canonical point y_c (Sec. 4.4);
                 canon = marked dilated by r cells: canon(c) = OR of marked(c')
                 over |c' - c|_inf <= r, c' inside the grid.
  posed          posed(c) = S(y_c) >= s_min and canon(clamp(floor((x_final - bmin) / h),
                 0, G - 1)), where S and x_final are the bone-weight sum of Eq. lbs
                 and the canonical point after MLP_res (Sec. 4.2, Sec. 4.3) with
                 every PE band on.

The cell test is the value at the centre; the dilation covers the points of a
cell, which a locally rigid warp moves by at most half a cell diagonal from the
centre's image, and the clamp keeps a cell whose centre maps just outside the
box (a canonical point there has no density) while others of its points map
inside.  Threshold, dilation and the weight floor s_min are parameters
(the paper gives no values).  Every step is the definition above written out
in float64, cell by cell.
"""
from __future__ import annotations

import numpy as np
import torch

from .field import F64, Params, canonical_mlp, hash_encode, residual_offset, skeleton_warp, t64


def cell_centres(box_min, box_max, grid: int) -> torch.Tensor:
    """Centres [G^3][3] in linear cell order (x fastest, then y, then z)."""
    bmin, bmax = t64(box_min), t64(box_max)
    h = (bmax - bmin) / grid
    j = torch.arange(grid, dtype=F64) + 0.5
    cz, cy, cx = torch.meshgrid(j, j, j, indexing="ij")
    return torch.stack([bmin[0] + cx.reshape(-1) * h[0], bmin[1] + cy.reshape(-1) * h[1],
                        bmin[2] + cz.reshape(-1) * h[2]], 1)


def canonical_sigma(P: Params, grid: int, chunk: int = 65536) -> torch.Tensor:
    """sigma [G^3] of the canonical field at every canonical cell centre."""
    y = cell_centres(P.box_min, P.box_max, grid)
    out = torch.empty(y.shape[0], dtype=F64)
    with torch.no_grad():
        for c0 in range(0, y.shape[0], chunk):
            enc, _ = hash_encode(y[c0:c0 + chunk], P.table, P.level_res, P.box_min, P.box_max)
            _, sigma = canonical_mlp(enc, P.mlp)
            out[c0:c0 + chunk] = sigma
    return out


def dilate(mask: np.ndarray, grid: int, r: int) -> np.ndarray:
    """OR of mask over the (2r+1)^3 neighbourhood of each cell, clipped at the grid's faces.

    mask: bool [G^3] in linear cell order; returns the same layout.
    """
    m = np.asarray(mask, bool).reshape(grid, grid, grid)      # [z][y][x]
    out = np.zeros_like(m)
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                # out[z, y, x] |= m[z + dz, y + dy, x + dx] where the neighbour exists
                src = m[max(dz, 0):grid + min(dz, 0), max(dy, 0):grid + min(dy, 0), max(dx, 0):grid + min(dx, 0)]
                out[max(-dz, 0):grid + min(-dz, 0), max(-dy, 0):grid + min(-dy, 0),
                    max(-dx, 0):grid + min(-dx, 0)] |= src
    return out.reshape(-1)


def canonical_grid(P: Params, grid: int, tau: float, r: int):
    """(canon bool [G^3], sigma [G^3]): the dilated canonical occupancy and the densities it came from."""
    sigma = canonical_sigma(P, grid)
    return dilate((sigma > tau).numpy(), grid, r), sigma


def posed_points(P: Params, G_R, G_t, omega, grid: int, chunk: int = 65536):
    """(S [G^3], x_final [G^3][3]) at every observed cell centre for one pose."""
    y = cell_centres(P.box_min, P.box_max, grid)
    S = torch.empty(y.shape[0], dtype=F64)
    xf = torch.empty_like(y)
    with torch.no_grad():
        for c0 in range(0, y.shape[0], chunk):
            x_skel, s = skeleton_warp(y[c0:c0 + chunk], G_R, G_t, P.wvol, P.box_min, P.box_max)
            if P.res_enabled:
                x_skel = x_skel + residual_offset(x_skel, omega, P.res, P.box_min, P.box_max, P.res_freqs)
            S[c0:c0 + chunk] = s
            xf[c0:c0 + chunk] = x_skel
    return S, xf


def canonical_cell(x_final: torch.Tensor, box_min, box_max, grid: int):
    """(cell index [N] clamped to the grid, position [N][3] in cell units)."""
    bmin, bmax = t64(box_min), t64(box_max)
    u = (x_final - bmin) / ((bmax - bmin) / grid)
    ci = torch.floor(u).clamp(0, grid - 1).to(torch.int64)
    return (ci[:, 2] * grid + ci[:, 1]) * grid + ci[:, 0], u


def posed_grid(canon: np.ndarray, S: torch.Tensor, x_final: torch.Tensor, box_min, box_max, grid: int,
               s_min: float) -> np.ndarray:
    """posed bool [G^3] from the canonical grid and the warped cell centres."""
    idx, _ = canonical_cell(x_final, box_min, box_max, grid)
    return np.asarray(canon, bool)[idx.numpy()] & (S.numpy() >= s_min)


def pack(mask: np.ndarray) -> np.ndarray:
    """bool [G^3] -> uint32 words, cell c at bit c & 31 of word c >> 5."""
    m = np.asarray(mask, bool).reshape(-1, 32).astype(np.uint64)
    return (m << np.arange(32, dtype=np.uint64)).sum(1).astype(np.uint32)


def unpack(words: np.ndarray) -> np.ndarray:
    w = np.asarray(words, np.uint32)
    return ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool).reshape(-1)
