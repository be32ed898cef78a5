"""The per-point field of the dynamic human (oracle, FP64, plain PyTorch CPU ops).

Test infrastructure: only tests, smoke() and the bench's CPU-baseline leg use it.

For an observation-space point x and the observed pose theta^o, Sec. 4 gives

    x_skel  = M_skel(x, theta^o) = sum_i w_i^o(x) G_i(x)              (Sec. 4.2)
    w_i^o   = w_i^c(G_i x) / sum_k w_k^c(G_k x)                      (Sec. 4.2, Eq. lbs)
    x_res   = MLP_res(gamma(x_skel), Omega^o)                         (Sec. 4.3)
    x_final = x_skel + x_res                                          (Sec. 4.3)
    c, sigma = MLP_nerf(enc(x_final))                                 (Sec. 4.4)

and the likelihood of being on the performer is the denominator of Eq. lbs
(Sec. 4.4).  Every function below is one of these steps, written in the
paper's order, in float64, with no blocking or fusion.  Parameters are the
float32 values the renderer holds, widened to float64.

Readings of points the paper leaves open (each listed in the design notes):
  * w_i^c(G_i x) is channel i of the canonical weight volume sampled
    trilinearly at the candidate point p_i = G_i x; vertices are aligned with
    the box corners and a corner outside the volume contributes zero.
  * the denominator is clamped below: x_skel = sum w~_i p_i / max(S, 1e-4).
  * gamma(x) = [x^, sin(2^k pi x^), cos(2^k pi x^) for k < L], x^ the point
    normalised to [-1, 1] over the box, each band k scaled by the truncated
    Hann weight (1 - cos(pi clamp(a - k, 0, 1))) / 2 (Sec. 4.3).
  * the pose Omega^o (24 x 3 axis-angle) joins gamma at the first layer; the
    fourth layer sees [h3, gamma] (Fig. S3).
  * the canonical encoding is a multiresolution hash grid (the workloads fix
    it): per level, 8-corner trilinear interpolation of F features, dense
    row-major indexing where (N+1)^3 <= T, else the spatial hash
    (x * 1 ^ y * 2654435761 ^ z * 805459861) mod T; features are zero-padded
    to the MLP input width.
  * outputs: rgb = sigmoid(o[0:3]), sigma = softplus(o[3]).
  * a canonical point outside the box has no density.
"""
from __future__ import annotations

import math

import torch

F64 = torch.float64
EPS_W = 1e-4
PRIME_Y = 2654435761
PRIME_Z = 805459861


def t64(a) -> torch.Tensor:
    return torch.as_tensor(a).to(F64) if not isinstance(a, torch.Tensor) else a.to(F64)


# ---------------------------------------------------------------- Sec. 4.2

def trilinear_volume(vol: torch.Tensor, p: torch.Tensor, box_min, box_max) -> torch.Tensor:
    """Trilinear sample of one channel vol [R][R][R] (indexed [z][y][x]) at points p [N][3].

    Vertex (i, j, k) lies at box_min + (i, j, k) * (box_max - box_min) / (R - 1); a corner
    outside the grid contributes zero.
    """
    R = vol.shape[0]
    bmin, bmax = t64(box_min), t64(box_max)
    u = (p - bmin) / ((bmax - bmin) / (R - 1))
    i0 = torch.floor(u)
    f = u - i0
    i0 = i0.to(torch.int64)
    flat = vol.reshape(-1)
    out = torch.zeros(p.shape[0], dtype=F64)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                ix, iy, iz = i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz
                w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                     * (f[:, 2] if dz else 1 - f[:, 2]))
                ok = (ix >= 0) & (ix < R) & (iy >= 0) & (iy < R) & (iz >= 0) & (iz < R)
                idx = (iz.clamp(0, R - 1) * R + iy.clamp(0, R - 1)) * R + ix.clamp(0, R - 1)
                out = out + torch.where(ok, w * flat[idx], torch.zeros((), dtype=F64))
    return out


def skeleton_warp(x: torch.Tensor, G_R: torch.Tensor, G_t: torch.Tensor, wvol: torch.Tensor,
                  box_min, box_max):
    """Inverse LBS of observation points x [N][3] (Sec. 4.2).

    Returns (x_skel [N][3], S [N]) where S = sum_i w_i^c(G_i x) over the bone
    channels (the background channel, last, is not a bone).
    """
    K = G_R.shape[0]
    num = torch.zeros_like(x)
    S = torch.zeros(x.shape[0], dtype=F64)
    for i in range(K):
        p = x @ G_R[i].T + G_t[i]                     # G_i(x) = R_i x + t_i
        w = trilinear_volume(wvol[i], p, box_min, box_max)
        num = num + w[:, None] * p
        S = S + w
    x_skel = num / torch.clamp(S, min=EPS_W)[:, None]
    return x_skel, S


# ---------------------------------------------------------------- Sec. 4.3

def hann_weights(n_freqs: int, alpha: float) -> torch.Tensor:
    """Truncated Hann window over frequency bands: (1 - cos(pi clamp(alpha - k, 0, 1))) / 2."""
    k = torch.arange(n_freqs, dtype=F64)
    a = torch.clamp(alpha - k, 0.0, 1.0)
    return (1.0 - torch.cos(math.pi * a)) / 2.0


def positional_encoding(x: torch.Tensor, box_min, box_max, n_freqs: int, alpha: float | None = None):
    """gamma(x) = [x^, w_k sin(2^k pi x^), w_k cos(2^k pi x^)]_k on box-normalised x^ (3 + 6L dims)."""
    bmin, bmax = t64(box_min), t64(box_max)
    xh = (x - (bmin + bmax) / 2) / ((bmax - bmin) / 2)
    w = hann_weights(n_freqs, n_freqs if alpha is None else alpha)
    parts = [xh]
    for k in range(n_freqs):
        a = (2.0 ** k) * math.pi * xh
        parts.append(w[k] * torch.sin(a))
        parts.append(w[k] * torch.cos(a))
    return torch.cat(parts, dim=1)


def residual_offset(x_skel, omega, res_layers, box_min, box_max, n_freqs, alpha=None):
    """x_res = MLP_res(gamma(x_skel), Omega^o): 5 layers, ReLU, skip of gamma into layer 4 (Fig. S3)."""
    g = positional_encoding(x_skel, box_min, box_max, n_freqs, alpha)
    om = t64(omega).reshape(1, -1).expand(x_skel.shape[0], -1)
    (W1, b1), (W2, b2), (W3, b3), (W4, b4), (W5, b5) = res_layers
    h = torch.relu(torch.cat([g, om], 1) @ W1.T + b1)
    h = torch.relu(h @ W2.T + b2)
    h = torch.relu(h @ W3.T + b3)
    h = torch.relu(torch.cat([h, g], 1) @ W4.T + b4)
    return h @ W5.T + b5


# ---------------------------------------------------------------- Sec. 4.4

def level_is_dense(n: int, T: int) -> bool:
    return (n + 1) ** 3 <= T


def corner_index(ix, iy, iz, n: int, T: int) -> torch.Tensor:
    """Table slot of integer vertex (ix, iy, iz) on a level of resolution n with T slots."""
    if level_is_dense(n, T):
        return ix + iy * (n + 1) + iz * (n + 1) * (n + 1)
    m = 0xFFFFFFFF
    h = (ix & m) ^ ((iy * PRIME_Y) & m) ^ ((iz * PRIME_Z) & m)
    return h % T


def hash_encode(x: torch.Tensor, table: torch.Tensor, level_res, box_min, box_max):
    """Multiresolution hash encoding of canonical points x [N][3]: [N][L*F] and the inside mask.

    p = (x - box_min) / (box_max - box_min); on level l the point sits at p * N_l among vertices
    0..N_l; its cell is the floor of that, capped at N_l - 1.  Points outside the box get zeros.
    """
    bmin, bmax = t64(box_min), t64(box_max)
    p = (x - bmin) / (bmax - bmin)
    inside = ((p >= 0) & (p <= 1)).all(1)
    pc = torch.clamp(p, 0.0, 1.0)
    L, T, F = table.shape
    feats = []
    for l in range(L):
        n = int(level_res[l])
        pos = pc * n
        i0 = torch.clamp(torch.floor(pos), max=n - 1)
        f = pos - i0
        i0 = i0.to(torch.int64)
        acc = torch.zeros(x.shape[0], F, dtype=F64)
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                         * (f[:, 2] if dz else 1 - f[:, 2]))
                    idx = corner_index(i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz, n, T)
                    acc = acc + w[:, None] * table[l][idx]
        feats.append(acc)
    enc = torch.cat(feats, 1) * inside[:, None].to(F64)
    return enc, inside


def canonical_mlp(enc: torch.Tensor, layers):
    """MLP_nerf: ReLU hidden layers, linear output o[4]; rgb = sigmoid(o[:3]), sigma = softplus(o[3])."""
    mlp_in = layers[0][0].shape[1]
    h = enc
    if h.shape[1] < mlp_in:
        h = torch.cat([h, torch.zeros(h.shape[0], mlp_in - h.shape[1], dtype=F64)], 1)
    for W, b in layers[:-1]:
        h = torch.relu(h @ W.T + b)
    W, b = layers[-1]
    o = h @ W.T + b
    rgb = torch.sigmoid(o[:, :3])
    sigma = torch.clamp(o[:, 3], min=0) + torch.log1p(torch.exp(-torch.abs(o[:, 3])))
    return rgb, sigma


# ---------------------------------------------------------------- the chain

class Params:
    """The trainable parameters of one subject as float64 tensors (leaf tensors for autograd)."""

    def __init__(self, subj: dict, requires_grad: bool = False):
        rg = requires_grad
        self.wvol = t64(subj["wvol"]).clone().requires_grad_(rg)
        self.table = t64(subj["hash_table"]).clone().requires_grad_(rg)
        self.mlp = [(t64(W).clone().requires_grad_(rg), t64(b).clone().requires_grad_(rg))
                    for W, b in subj["mlp_layers"]]
        self.res = [(t64(W).clone().requires_grad_(rg), t64(b).clone().requires_grad_(rg))
                    for W, b in subj["res_layers"]]
        self.box_min = t64(subj["box_min"])
        self.box_max = t64(subj["box_max"])
        self.level_res = [int(v) for v in subj["level_res"]]
        self.res_enabled = bool(subj.get("res_enabled", 1))
        self.res_freqs = int(subj["res_pe_freqs"])

    def tensors(self):
        out = [self.wvol, self.table]
        for W, b in self.mlp + self.res:
            out += [W, b]
        return out


def field(x: torch.Tensor, P: Params, G_R, G_t, omega, alpha=None):
    """The whole per-point chain for observation points x [N][3].

    Returns dict(rgb [N][3], sigma [N], S [N], inside [N], x_skel, x_final).
    """
    x_skel, S = skeleton_warp(x, G_R, G_t, P.wvol, P.box_min, P.box_max)
    if P.res_enabled:
        x_final = x_skel + residual_offset(x_skel, omega, P.res, P.box_min, P.box_max,
                                           P.res_freqs, alpha)
    else:
        x_final = x_skel
    enc, inside = hash_encode(x_final, P.table, P.level_res, P.box_min, P.box_max)
    rgb, sigma = canonical_mlp(enc, P.mlp)
    return dict(rgb=rgb, sigma=sigma, S=S, inside=inside, x_skel=x_skel, x_final=x_final, enc=enc)
