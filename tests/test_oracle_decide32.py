"""Pins of the oracle's float32 occupancy decisions (Sec. 2.3 empty-space skipping).

`decide32.sample_points32` (bin midpoints, Sec. 2.1 Eq. 3 read with midpoint
samples) and `decide32.cell_of32` (cell, clamp and linear index of a sample)
decide which samples the oracle counts as live.  They are checked here against
quantities computed another way:
  - the midpoints against the FP64 points o + (lo + (i + 1/2) D) d;
  - the cells against an FP64 floor of the same points (points kept at least
    1e-4 cell away from every face), and against the clamp at the faces;
  - the axis order of the linear index against the posed bitfield's own
    meshgrid ordering (a separately written producer of the same words);
  - the skip end to end: an all-ones bitfield renders like no skipping at all,
    an all-zeros one gives the background.
"""
import numpy as np
import torch

from oracle import decide32
from oracle import field as OF
from oracle import render as OR
from paper_2306_16541_gb300 import synth

f32 = np.float32


def _rays(n=400, seed=3):
    cfg = synth.config_tiny()
    cam = cfg["camera"]
    s = cfg["subject"]
    g = np.random.default_rng(seed)
    px = g.integers(0, cam.width, n)
    py = g.integers(0, cam.height, n)
    o, d = decide32.ray_dirs32(cam, px, py)
    lo, hi, hit = decide32.clip32(o, d, cam.t_near, cam.t_far, s["box_min"], s["box_max"])
    return cfg, o[hit] if o.ndim == 2 else o, d[hit], lo[hit], hi[hit]


def test_sample_points_are_bin_midpoints():
    cfg, o, d, lo, hi = _rays()
    S = 32
    x = decide32.sample_points32(o, d, lo, hi, S)
    assert x.dtype == np.float32 and x.shape == (d.shape[0], S, 3)
    o64 = np.asarray(o, np.float64)
    d64, lo64, hi64 = d.astype(np.float64), lo.astype(np.float64), hi.astype(np.float64)
    D = (hi64 - lo64) / S
    t = lo64[:, None] + (np.arange(S)[None, :] + 0.5) * D[:, None]
    ref = o64[None, None, :] + t[:, :, None] * d64[:, None, :]
    # a handful of float32 roundings on numbers below 4 in magnitude
    err = np.abs(x.astype(np.float64) - ref)
    assert err.max() < 16 * np.finfo(np.float32).eps * 4.0
    # the bins' starts (i instead of i + 1/2) sit D/2 ~ 3 cm away: far outside that bound
    start = o64[None, None, :] + (lo64[:, None] + np.arange(S)[None, :] * D[:, None])[:, :, None] * d64[:, None, :]
    assert np.abs(x.astype(np.float64) - start).max() > 1e-3
    # consecutive samples are D apart along the unit direction
    step = np.linalg.norm(np.diff(x.astype(np.float64), axis=1), axis=2)
    assert np.allclose(step, D[:, None], atol=1e-5)


def test_cell_index_matches_fp64_floor_away_from_faces():
    g = np.random.default_rng(5)
    bmin = np.array([-1.0, -1.1, -0.9], f32)
    bmax = np.array([1.0, 0.9, 1.1], f32)
    G = 16
    x = g.uniform(bmin, bmax, size=(20000, 3)).astype(f32)
    h64 = (bmax.astype(np.float64) - bmin) / G
    u = (x.astype(np.float64) - bmin) / h64
    keep = (np.abs(u - np.round(u)) > 1e-4).all(1)
    x, u = x[keep], u[keep]
    c = np.floor(u).astype(np.int64)
    ref = (c[:, 2] * G + c[:, 1]) * G + c[:, 0]
    got = decide32.cell_of32(x, bmin, bmax, G)
    assert np.array_equal(got, ref)
    # each axis has its own stride: moving one cell along x, y, z changes the index by 1, G, G^2
    centre = (bmin + (np.array([3, 7, 11]) + 0.5) * h64).astype(f32)
    base = decide32.cell_of32(centre, bmin, bmax, G)
    assert base == (11 * G + 7) * G + 3
    for k, stride in enumerate([1, G, G * G]):
        y = centre.copy()
        y[k] = f32(y[k] + h64[k])
        assert decide32.cell_of32(y, bmin, bmax, G) - base == stride


def test_cell_index_clamps_at_the_faces():
    bmin = np.array([-1.0, -1.0, -1.0], f32)
    bmax = np.array([1.0, 1.0, 1.0], f32)
    G = 8
    pts = np.array([[-1.0, -1.0, -1.0],          # the minimum corner: cell 0
                    [1.0, 1.0, 1.0],             # the maximum corner: clamped into the last cell
                    [-1.5, 0.1, 2.0],            # outside on two axes: clamped per axis
                    [0.999999, -0.999999, 0.0]], f32)
    got = decide32.cell_of32(pts, bmin, bmax, G)
    h = 2.0 / G
    def lin(cx, cy, cz):
        return (cz * G + cy) * G + cx
    assert got[0] == 0
    assert got[1] == lin(G - 1, G - 1, G - 1)
    assert got[2] == lin(0, int(np.floor((0.1 + 1.0) / h)), G - 1)
    assert got[3] == lin(G - 1, 0, G // 2)
    assert (got >= 0).all() and (got < G ** 3).all()


def test_cell_order_agrees_with_the_bitfield_producer():
    # posed_bitfield32 lays its cells out with a (z, y, x) meshgrid; one small ellipsoid at an
    # off-diagonal point must be found by cell_of32 at that point and not at its axis swaps
    G = 16
    bmin, bmax = [-1.0] * 3, [1.0] * 3
    p = np.array([0.55, -0.3, 0.1], f32)
    E = np.zeros((1, 15), f32)
    E[0, :3] = p
    E[0, 3:12] = np.eye(3, dtype=f32).ravel()
    E[0, 12:15] = 0.01
    G_id = np.zeros((1, 12), f32)
    G_id[0, [0, 5, 10]] = 1.0
    bits = decide32.posed_bitfield32(G_id, E, bmin, bmax, G)
    assert decide32.bit_test(bits, decide32.cell_of32(p, bmin, bmax, G))
    for perm in ([1, 0, 2], [2, 1, 0], [0, 2, 1]):
        q = p[perm]
        assert not decide32.bit_test(bits, decide32.cell_of32(q, bmin, bmax, G))
    # the set cells are exactly the cells whose centre lies within half a diagonal of p
    n_set = int(sum(bin(int(w)).count("1") for w in bits))
    h = 2.0 / G
    j = (np.arange(G) + 0.5) * h - 1.0
    cz, cy, cx = np.meshgrid(j, j, j, indexing="ij")
    dist = np.sqrt((cx - p[0]) ** 2 + (cy - p[1]) ** 2 + (cz - p[2]) ** 2)
    near = dist <= 0.01 + 0.5 * np.sqrt(3) * h
    assert n_set == int(near.sum())


def _render(cfg, use_occ, bits=None, n=300):
    s = cfg["subject"]
    cam = cfg["camera"]
    g = np.random.default_rng(9)
    px = g.integers(0, cam.width, n)
    py = g.integers(0, cam.height, n)
    P = OF.Params(s)
    out, counts = OR.render_pixels(s, P, cfg["pose"], cam, px, py, use_occ, grid=32, bits=bits,
                                   return_counts=True)
    return out.numpy(), counts, cam


def test_all_ones_bitfield_renders_like_no_skipping():
    cfg = synth.config_tiny()
    cfg["subject"] = synth.subject(1234, hash_scale=0.5, res_last_std=0.02)
    ones = np.full(32 ** 3 // 32, 0xFFFFFFFF, np.uint32)
    a, ca, _ = _render(cfg, True, ones)
    b, cb, _ = _render(cfg, False)
    assert np.array_equal(a, b)
    assert np.array_equal(ca, cb)
    assert (ca > 0).any()


def test_all_zeros_bitfield_gives_the_background():
    cfg = synth.config_tiny()
    cfg["subject"] = synth.subject(1234, hash_scale=0.5, res_last_std=0.02)
    cfg["camera"].bg = np.array([0.25, 0.5, 0.75], f32)
    zeros = np.zeros(32 ** 3 // 32, np.uint32)
    out, counts, cam = _render(cfg, True, zeros)
    assert (counts == 0).all()
    bg = np.asarray(cam.bg, np.float64)
    assert np.array_equal(out[:, :3], np.broadcast_to(bg.astype(np.float32).astype(np.float64), out[:, :3].shape))
    assert (out[:, 3] == 0).all()
    # without skipping the same pixels are not all background
    b, _, _ = _render(cfg, False)
    assert np.abs(b[:, :3] - out[:, :3]).max() > 1e-3
