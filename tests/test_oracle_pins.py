"""Pins of the FP64 oracle against things other than itself.

Closed forms of Eq. 2-3 (Sec. 2.1), invariants of inverse LBS (Sec. 4.2),
library routines (grid_sample, numpy matmul, torch.optim.Adam), the published
SplitMix64 test vector, exactness properties of the hash encoding, and a
scalar brute-force expansion of the whole chain on a tiny subject.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import decide32, fk, rng
from oracle import field as OF
from oracle import render as OR
from paper_2306_16541_gb300 import synth

F64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ compositing (Eq. 2-3)

def test_constant_density_transmittance_closed_form():
    # constant sigma over a ray of length L: T_final = exp(-sigma L), sum w = 1 - T_final
    sigma, L, S = 0.7, 2.0, 64
    lo = torch.tensor([1.5], dtype=F64)
    hi = lo + L
    t, delta = OR.sample_t(lo, hi, S)
    alpha = 1.0 - torch.exp(-sigma * delta)
    c = torch.tensor([0.2, 0.5, 0.9], dtype=F64)
    bg = np.array([0.3, 0.1, 0.7])
    rgba, w = OR.composite(c.expand(1, S, 3), alpha, bg)
    Tf = math.exp(-sigma * L)
    assert abs((1 - rgba[0, 3].item()) - Tf) < 1e-14
    assert abs(w.sum().item() - (1 - Tf)) < 1e-14
    expect = c * (1 - Tf) + torch.tensor(bg) * Tf
    assert torch.allclose(rgba[0, :3], expect, atol=1e-14, rtol=0)


def test_stratified_spacing_sums_to_ray_length():
    lo = torch.tensor([0.5, 1.0], dtype=F64)
    hi = torch.tensor([3.0, 1.25], dtype=F64)
    u = rng.jitter(7, 2, 16)
    t, delta = OR.sample_t(lo, hi, 16, u)
    assert torch.allclose(delta.sum(1) + (t[:, 0] - lo), hi - lo, atol=1e-14)
    assert (delta > 0).all()
    bins = (t - lo[:, None]) / ((hi - lo) / 16)[:, None]
    assert ((bins - torch.arange(16)) >= 0).all() and ((bins - torch.arange(16)) < 1).all()


def test_weights_bounded_and_alpha_cap():
    g = torch.Generator().manual_seed(0)
    a = torch.rand(50, 20, generator=g, dtype=F64)
    rgb = torch.rand(50, 20, 3, generator=g, dtype=F64)
    rgba, w = OR.composite(rgb, a, np.zeros(3))
    assert (w >= 0).all() and (w.sum(1) <= 1 + 1e-15).all()
    assert torch.allclose(w.sum(1), rgba[:, 3], atol=1e-14)


def test_likelihood_augmentation_caps_alpha():
    # alpha_i = (1 - exp(-sigma delta)) * min(S, 1): S >= 1 leaves it, S -> 0 suppresses it (Sec. 4.4)
    out = dict(sigma=torch.tensor([2.0, 2.0, 2.0], dtype=F64), S=torch.tensor([1.7, 0.25, 0.0], dtype=F64),
               inside=torch.tensor([True, True, True]))
    a = OR.sample_alpha(out, torch.tensor([0.1, 0.1, 0.1], dtype=F64), torch.tensor([True, True, True]))
    base = 1 - math.exp(-0.2)
    assert torch.allclose(a, torch.tensor([base, 0.25 * base, 0.0], dtype=F64), atol=1e-15)


# ------------------------------------------------------------ LBS warp (Sec. 4.2)

def test_trilinear_matches_grid_sample():
    g = torch.Generator().manual_seed(1)
    R = 9
    vol = torch.rand(R, R, R, generator=g, dtype=F64)
    p = (torch.rand(2000, 3, generator=g, dtype=F64) * 2.4 - 1.2)        # some points outside
    got = OF.trilinear_volume(vol, p, [-1, -1, -1], [1, 1, 1])
    ref = torch.nn.functional.grid_sample(vol[None, None], p[None, :, None, None, :], mode="bilinear",
                                          padding_mode="zeros", align_corners=True)[0, 0, :, 0, 0]
    assert torch.allclose(got, ref, atol=1e-13, rtol=0)


def _identity_G(K):
    return torch.eye(3, dtype=F64).expand(K, 3, 3).clone(), torch.zeros(K, 3, dtype=F64)


def test_rest_pose_warp_is_identity():
    subj = synth.subject(5)
    vol = OF.t64(subj["wvol"])
    R, t = fk.bone_transforms(subj["parents"], subj["rest_joints"], np.zeros((24, 3)), np.zeros(3))
    assert np.allclose(R, np.eye(3)) and np.allclose(t, 0, atol=1e-15)
    g = torch.Generator().manual_seed(2)
    x = torch.rand(500, 3, generator=g, dtype=F64) * 1.6 - 0.8
    xs, S = OF.skeleton_warp(x, torch.from_numpy(R), torch.from_numpy(t), vol, subj["box_min"], subj["box_max"])
    m = S > OF.EPS_W
    assert m.sum() > 100
    assert torch.allclose(xs[m], x[m], atol=1e-12)


def test_one_hot_volume_gives_rigid_transform():
    K, R_ = 3, 8
    vol = torch.zeros(K + 1, R_, R_, R_, dtype=F64)
    vol[1] = 1.0
    aa = np.array([[0.1, 0.2, 0.3], [0.3, -0.2, 0.25], [0.0, 0.4, -0.1]])
    R, t = fk.bone_transforms(np.array([-1, 0, 1]), np.array([[0, 0, 0], [0, 0.3, 0], [0, 0.6, 0.0]]),
                              aa, np.array([0.05, 0.0, 0.0]))
    g = torch.Generator().manual_seed(3)
    x = torch.rand(200, 3, generator=g, dtype=F64) * 0.4 - 0.2
    xs, S = OF.skeleton_warp(x, torch.from_numpy(R), torch.from_numpy(t), vol, [-1] * 3, [1] * 3)
    expect = x @ torch.from_numpy(R[1]).T + torch.from_numpy(t[1])
    assert torch.allclose(S, torch.ones_like(S), atol=1e-14)
    assert torch.allclose(xs, expect, atol=1e-14)


def test_observation_weights_sum_to_one():
    subj = synth.subject(6)
    aa, rt = synth.random_pose(np.random.default_rng(0))
    R, t = fk.bone_transforms(subj["parents"], subj["rest_joints"], aa, rt)
    vol = OF.t64(subj["wvol"])
    x = torch.rand(300, 3, dtype=F64, generator=torch.Generator().manual_seed(4)) * 1.4 - 0.7
    ws = []
    for i in range(24):
        p = x @ torch.from_numpy(R[i]).T + torch.from_numpy(t[i])
        ws.append(OF.trilinear_volume(vol[i], p, subj["box_min"], subj["box_max"]))
    w = torch.stack(ws, 1)
    S = w.sum(1)
    m = S > 1e-3
    assert torch.allclose((w[m] / S[m, None]).sum(1), torch.ones(int(m.sum()), dtype=F64), atol=1e-13)


# ------------------------------------------------------------ forward kinematics

def test_fk_chain_against_direct_products():
    parents = np.array([-1, 0, 1])
    J = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.0], [0.0, 1.0, 0.0]])
    aa = np.array([[0.0, 0.0, math.pi / 2], [0.0, 0.0, math.pi / 2], [0.0, 0.0, 0.0]])
    AR, At = fk.posed_joints(parents, J, aa, np.array([1.0, 0.0, 0.0]))
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    assert np.allclose(AR[1], Rz @ Rz)
    # joint 1 sits at root + Rz (0, .5, 0) = (1 - .5, 0, 0); joint 2 = joint1 + Rz Rz (0, .5, 0)
    assert np.allclose(At[1], [0.5, 0.0, 0.0])
    assert np.allclose(At[2], [0.5, -0.5, 0.0])
    R, t = fk.bone_transforms(parents, J, aa, np.array([1.0, 0.0, 0.0]))
    for i in range(3):                       # G_i maps the posed joint back to its rest position
        assert np.allclose(R[i] @ At[i] + t[i], J[i])
    assert np.allclose(fk.rodrigues(np.array([0.0, 0.0, math.pi / 2])), Rz)


def test_rodrigues_is_a_rotation_and_matches_series():
    aa = np.random.default_rng(0).normal(size=(20, 3)) * 0.5
    Rm = fk.rodrigues(aa)
    for a, R in zip(aa, Rm):
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
        E = np.eye(3)
        term = np.eye(3)
        for n in range(1, 30):                   # matrix exponential by its power series
            term = term @ K / n
            E = E + term
        assert np.allclose(R, E, atol=1e-13)


# ------------------------------------------------------------ positional encoding, Hann window (Sec. 4.3)

def test_positional_encoding_values():
    x = torch.tensor([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]], dtype=F64)
    g = OF.positional_encoding(x, [-1] * 3, [1] * 3, 3)
    assert g.shape == (2, 3 + 18)
    assert torch.allclose(g[0], torch.tensor([0, 0, 0] + [0, 0, 0, 1, 1, 1] * 3, dtype=F64), atol=1e-15)
    expect = [0.5] * 3 + [1, 1, 1, 0, 0, 0] + [0, 0, 0, -1, -1, -1] + [0, 0, 0, 1, 1, 1]
    assert torch.allclose(g[1], torch.tensor(expect, dtype=F64), atol=1e-14)


def test_hann_window():
    assert torch.allclose(OF.hann_weights(6, 0.0), torch.zeros(6, dtype=F64))
    assert torch.allclose(OF.hann_weights(6, 6.0), torch.ones(6, dtype=F64))
    w = OF.hann_weights(6, 2.5)
    assert torch.allclose(w, torch.tensor([1, 1, 0.5, 0, 0, 0], dtype=F64), atol=1e-15)


# ------------------------------------------------------------ hash encoding

def test_hash_exact_at_vertices_and_linear_on_dense_level():
    L, T = 2, 4096
    levels = [7, 40]                       # 8^3 = 512 <= T dense; 41^3 > T hashed
    g = torch.Generator().manual_seed(5)
    table = torch.rand(L, T, 2, generator=g, dtype=F64)
    # dense level 0 holds a linear function of the vertex coordinates
    n = levels[0]
    iz, iy, ix = torch.meshgrid(torch.arange(n + 1), torch.arange(n + 1), torch.arange(n + 1), indexing="ij")
    idx = OF.corner_index(ix.reshape(-1), iy.reshape(-1), iz.reshape(-1), n, T)
    lin = 0.3 * ix + 0.7 * iy - 0.2 * iz + 1.0
    table[0, idx, 0] = lin.reshape(-1).to(F64)
    table[0, idx, 1] = -lin.reshape(-1).to(F64)
    x = torch.rand(300, 3, generator=g, dtype=F64) * 2 - 1
    enc, inside = OF.hash_encode(x, table, levels, [-1] * 3, [1] * 3)
    p = (x + 1) / 2 * n
    expect = 0.3 * p[:, 0] + 0.7 * p[:, 1] - 0.2 * p[:, 2] + 1.0
    assert inside.all()
    assert torch.allclose(enc[:, 0], expect, atol=1e-12) and torch.allclose(enc[:, 1], -expect, atol=1e-12)
    # at a vertex of the hashed level the encoding is that vertex's slot
    n1 = levels[1]
    v = torch.tensor([[3, 17, 29], [0, 0, 0], [40, 40, 40], [11, 2, 39]])
    xv = v.to(F64) / n1 * 2 - 1
    enc, _ = OF.hash_encode(xv, table, levels, [-1] * 3, [1] * 3)
    for r in range(v.shape[0]):
        a, b, c = (int(q) for q in v[r])
        slot = ((a * 1) ^ ((b * 2654435761) & 0xFFFFFFFF) ^ ((c * 805459861) & 0xFFFFFFFF)) % T
        assert torch.allclose(enc[r, 2:4], table[1, slot], atol=1e-12)


def test_hash_index_brute_force_tiny_table():
    T, n = 16, 5
    for (a, b, c) in [(0, 0, 0), (1, 2, 3), (5, 5, 5), (4, 0, 1), (2, 3, 0)]:
        brute = 0
        for bit in range(32):                   # xor built bit by bit from the products
            pa, pb, pc = a, (b * 2654435761) % 2 ** 32, (c * 805459861) % 2 ** 32
            brute |= (((pa >> bit) ^ (pb >> bit) ^ (pc >> bit)) & 1) << bit
        got = int(OF.corner_index(torch.tensor(a), torch.tensor(b), torch.tensor(c), n, T))
        assert got == brute % T
    assert not OF.level_is_dense(5, 16) and OF.level_is_dense(1, 8)


def test_level_resolutions_growth_rule():
    assert synth.level_resolutions(8, 16, 256) == [16, 23, 35, 52, 78, 115, 172, 256]
    assert synth.level_resolutions(16, 16, 2048) == [16, 22, 30, 42, 58, 80, 111, 153, 212, 294, 406,
                                                    561, 776, 1072, 1482, 2048]


def test_outside_box_has_no_features():
    table = torch.ones(2, 64, 2, dtype=F64)
    x = torch.tensor([[0.0, 0.0, 0.0], [1.01, 0.0, 0.0], [0.0, -1.2, 0.0]], dtype=F64)
    enc, inside = OF.hash_encode(x, table, [2, 5], [-1] * 3, [1] * 3)
    assert inside.tolist() == [True, False, False]
    assert torch.allclose(enc[0], torch.ones(4, dtype=F64)) and (enc[1:] == 0).all()


# ------------------------------------------------------------ MLPs

def test_canonical_mlp_matches_numpy():
    subj = synth.subject(9, hidden_layers=3)
    P = OF.Params(subj)
    x = np.random.default_rng(1).normal(size=(64, 32))
    rgb, sigma = OF.canonical_mlp(torch.from_numpy(x), P.mlp)
    h = x
    for W, b in subj["mlp_layers"][:-1]:
        h = np.maximum(h @ W.astype(np.float64).T + b, 0)
    W, b = subj["mlp_layers"][-1]
    o = h @ W.astype(np.float64).T + b
    assert np.allclose(rgb.numpy(), 1 / (1 + np.exp(-o[:, :3])), atol=1e-14)
    assert np.allclose(sigma.numpy(), np.log(1 + np.exp(o[:, 3])), atol=1e-13)


def test_residual_is_zero_at_init_and_skip_matters():
    subj = synth.subject(10)
    P = OF.Params(subj)
    x = torch.rand(32, 3, dtype=F64) - 0.5
    off = OF.residual_offset(x, np.zeros(72), P.res, P.box_min, P.box_max, 6)
    assert (off == 0).all()
    subj = synth.subject(10, res_last_std=0.01)
    P = OF.Params(subj)
    off = OF.residual_offset(x, np.zeros(72), P.res, P.box_min, P.box_max, 6)
    # numpy re-expansion with the skip concat at layer 4
    g = OF.positional_encoding(x, P.box_min, P.box_max, 6).numpy()
    Ls = [(W.astype(np.float64), b.astype(np.float64)) for W, b in subj["res_layers"]]
    h = np.maximum(np.concatenate([g, np.zeros((32, 72))], 1) @ Ls[0][0].T + Ls[0][1], 0)
    h = np.maximum(h @ Ls[1][0].T + Ls[1][1], 0)
    h = np.maximum(h @ Ls[2][0].T + Ls[2][1], 0)
    h = np.maximum(np.concatenate([h, g], 1) @ Ls[3][0].T + Ls[3][1], 0)
    assert np.allclose(off.numpy(), h @ Ls[4][0].T + Ls[4][1], atol=1e-14)
    assert off.abs().max() > 1e-4


# ------------------------------------------------------------ float32 decisions

def test_float32_rays_agree_with_fp64():
    cfg = synth.config_tiny()
    cam = cfg["camera"]
    py, px = np.meshgrid(np.arange(64), np.arange(64), indexing="ij")
    o32, d32 = decide32.ray_dirs32(cam, px.ravel(), py.ravel())
    o, d = OR.rays64(cam, px.ravel(), py.ravel())
    assert np.allclose(o32, o.numpy(), atol=1e-6) and np.allclose(d32, d.numpy(), atol=1e-6)
    lo, hi, hit = decide32.clip32(o32, d32, cam.t_near, cam.t_far, [-1] * 3, [1] * 3)
    c = 32 * 64 + 32
    # the ray through pixel (32, 32) runs near the optical axis: [1.5, 3.5] clipped by z = +-1
    assert abs(lo[c] - 1.5) < 1e-3 and abs(hi[c] - 3.5) < 1e-3 and hit.all()


def test_bitfield_matches_brute_force_point_test():
    E = np.zeros((1, 15), np.float32)
    E[0, :3] = [0.1, -0.2, 0.05]
    Q = fk.rodrigues(np.array([0.3, 0.2, -0.4]))
    E[0, 3:12] = Q.reshape(-1)
    E[0, 12:15] = [0.5, 0.2, 0.3]
    G = fk.bone_transforms_f32(np.array([-1]), np.zeros((1, 3)), np.array([[0.2, -0.1, 0.3]]), np.zeros(3))
    grid = 16
    bits = decide32.posed_bitfield32(G, E, [-1] * 3, [1] * 3, grid)
    h = 2.0 / grid
    dil = 0.5 * math.sqrt(3) * h
    Gm = G.reshape(3, 4).astype(np.float64)
    ok = 0
    for cz in range(grid):
        for cy in range(grid):
            for cx in range(grid):
                y = -1 + (np.array([cx, cy, cz]) + 0.5) * h
                q = Gm[:, :3] @ y + Gm[:, 3]
                s = ((Q @ (q - E[0, :3])) / (E[0, 12:15] + dil)) ** 2
                inside = s.sum() <= 1
                c = (cz * grid + cy) * grid + cx
                got = bool((bits[c >> 5] >> (c & 31)) & 1)
                if abs(s.sum() - 1) > 1e-4:       # away from the float32 rounding band
                    assert got == inside
                    ok += 1
    assert ok > grid ** 3 * 0.9 and bits.any()


def test_splitmix64_published_vector():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if not l.startswith("#")]
    seed = int(lines[0][1])
    expect = [int(l[0]) for l in lines[1:]]
    got = rng.splitmix64(seed, np.arange(1, 6, dtype=np.uint64))
    assert [int(v) for v in got] == expect
    u = rng.jitter(3, 4, 8)
    assert (u >= 0).all() and (u < 1).all() and u.dtype == np.float32


# ------------------------------------------------------------ brute force on a tiny subject

def _tiny_subject():
    r = np.random.default_rng(11)
    K = 2
    s = dict(parents=np.array([-1, 0], np.int32),
             rest_joints=np.array([[0.0, -0.2, 0.0], [0.0, 0.3, 0.0]], np.float32),
             box_min=np.array([-1, -1, -1], np.float32), box_max=np.array([1, 1, 1], np.float32),
             wvol=r.uniform(0.0, 0.6, size=(K + 1, 3, 3, 3)).astype(np.float32), wvol_res=3,
             level_res=np.array([1, 3], np.uint32), log2_T=4,
             hash_table=r.uniform(-1, 1, size=(2, 16, 2)).astype(np.float32),
             res_pe_freqs=1, res_enabled=1)
    s["mlp_layers"] = [(r.normal(size=(o, i)).astype(np.float32), r.normal(size=o).astype(np.float32) * 0.1)
                       for i, o in [(4, 4), (4, 4), (4, 4)]]
    s["res_layers"] = [(r.normal(size=(o, i)).astype(np.float32) * 0.3, r.normal(size=o).astype(np.float32) * 0.1)
                       for i, o in [(9 + 6, 4), (4, 4), (4, 4), (4 + 9, 4), (4, 3)]]
    return s


def _brute_pixel(s, cam, G, omega, u, v):
    """Scalar pure-Python expansion of one pixel (no vectorisation, no torch)."""
    def mv(M, x):
        return [sum(M[r][c] * x[c] for c in range(len(x))) for r in range(len(M))]
    R = [[float(q) for q in row] for row in cam.R]
    tt = [float(q) for q in cam.t]
    o = [-sum(R[r][k] * tt[r] for r in range(3)) for k in range(3)]
    a = [(u + 0.5 - cam.cx) / cam.fx, (v + 0.5 - cam.cy) / cam.fy, 1.0]
    w = [sum(R[r][k] * a[r] for r in range(3)) for k in range(3)]
    nrm = math.sqrt(sum(q * q for q in w))
    d = [q / nrm for q in w]
    lo, hi = cam.t_near, cam.t_far
    for k in range(3):
        ta, tb = (-1 - o[k]) / d[k], (1 - o[k]) / d[k]
        lo, hi = max(lo, min(ta, tb)), min(hi, max(ta, tb))
    bg = [float(q) for q in cam.bg]
    if not lo < hi:
        return bg + [0.0]
    S = cam.n_samples
    D = (hi - lo) / S
    vol = s["wvol"].astype(np.float64)
    Rv = vol.shape[1]
    T = 1.0
    C = [0.0, 0.0, 0.0]

    def tri(ch, p):
        uu = [(p[k] + 1) / (2 / (Rv - 1)) for k in range(3)]
        i0 = [math.floor(q) for q in uu]
        f = [uu[k] - i0[k] for k in range(3)]
        acc = 0.0
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    ix, iy, iz = i0[0] + dx, i0[1] + dy, i0[2] + dz
                    if 0 <= ix < Rv and 0 <= iy < Rv and 0 <= iz < Rv:
                        wt = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                        acc += wt * vol[ch, iz, iy, ix]
        return acc

    for i in range(S):
        t = lo + (i + 0.5) * D
        x = [o[k] + t * d[k] for k in range(3)]
        num, Ssum = [0.0] * 3, 0.0
        for b in range(2):
            p = [sum(G[b][0][r][c] * x[c] for c in range(3)) + G[b][1][r] for r in range(3)]
            wt = tri(b, p)
            Ssum += wt
            num = [num[k] + wt * p[k] for k in range(3)]
        xs = [q / max(Ssum, 1e-4) for q in num]
        gam = list(xs) + [math.sin(math.pi * q) for q in xs] + [math.cos(math.pi * q) for q in xs]
        Ls = [(W.astype(np.float64).tolist(), b.astype(np.float64).tolist()) for W, b in s["res_layers"]]
        h = [max(0.0, q + bb) for q, bb in zip(mv(Ls[0][0], gam + list(omega)), Ls[0][1])]
        h = [max(0.0, q + bb) for q, bb in zip(mv(Ls[1][0], h), Ls[1][1])]
        h = [max(0.0, q + bb) for q, bb in zip(mv(Ls[2][0], h), Ls[2][1])]
        h = [max(0.0, q + bb) for q, bb in zip(mv(Ls[3][0], h + gam), Ls[3][1])]
        xr = [q + bb for q, bb in zip(mv(Ls[4][0], h), Ls[4][1])]
        xf = [xs[k] + xr[k] for k in range(3)]
        pn = [(q + 1) / 2 for q in xf]
        inside = all(0 <= q <= 1 for q in pn)
        feats = []
        for l, n in enumerate([1, 3]):
            pos = [min(max(q, 0.0), 1.0) * n for q in pn]
            i0 = [min(math.floor(q), n - 1) for q in pos]
            f = [pos[k] - i0[k] for k in range(3)]
            acc = [0.0, 0.0]
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        cx, cy, cz = i0[0] + dx, i0[1] + dy, i0[2] + dz
                        if (n + 1) ** 3 <= 16:
                            slot = cx + cy * (n + 1) + cz * (n + 1) ** 2
                        else:
                            slot = (cx ^ ((cy * 2654435761) % 2 ** 32) ^ ((cz * 805459861) % 2 ** 32)) % 16
                        wt = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                        acc = [acc[j] + wt * float(s["hash_table"][l, slot, j]) for j in range(2)]
            feats += acc
        if not inside:
            feats = [0.0] * 4
        Ms = [(W.astype(np.float64).tolist(), b.astype(np.float64).tolist()) for W, b in s["mlp_layers"]]
        h = feats
        for W, b in Ms[:-1]:
            h = [max(0.0, q + bb) for q, bb in zip(mv(W, h), b)]
        out = [q + bb for q, bb in zip(mv(Ms[-1][0], h), Ms[-1][1])]
        rgb = [1 / (1 + math.exp(-q)) for q in out[:3]]
        sigma = math.log1p(math.exp(out[3]))
        alpha = (1 - math.exp(-sigma * D)) * min(Ssum, 1.0) if inside else 0.0
        C = [C[k] + T * alpha * rgb[k] for k in range(3)]
        T *= 1 - alpha
    return [C[k] + T * bg[k] for k in range(3)] + [1 - T]


def test_brute_force_tiny_chain():
    s = _tiny_subject()
    cam = synth.camera(2, 2, 2.0, (0.3, 0.2, 2.5), 3, 1.0, 4.0, bg=(0.1, 0.2, 0.3))
    aa = np.array([[0.1, -0.2, 0.15], [0.3, 0.1, -0.2]], np.float32)
    rt = np.array([0.02, -0.01, 0.0], np.float32)
    R, t = fk.bone_transforms(s["parents"], s["rest_joints"], aa, rt)
    G = [(R[b].tolist(), t[b].tolist()) for b in range(2)]
    P = OF.Params(s)
    got = OR.render_pixels(s, P, (aa, rt), cam, np.array([0, 1, 0, 1]), np.array([0, 0, 1, 1]), False)
    for r, (u, v) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
        ref = _brute_pixel(s, cam, G, aa.reshape(-1).astype(np.float64), u, v)
        assert np.allclose(got[r].numpy(), ref, atol=1e-12), (r, got[r], ref)
    assert (got[:, 3] > 0.05).any()
