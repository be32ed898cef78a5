"""Occupancy from the field's own density (Sec. 2.3 empty-space skipping for a
subject without ellipsoids): the canonical refresh, its posing through the
warp, rendering with it, and that skipping with it leaves the image unchanged.

The refresh and the posing decide bits from float32 values (a density against
its threshold, a warped point against a cell face).  The oracle decides them in
float64; a cell whose float64 value lies within a rounding band of the decision
boundary may go either way, and the test accepts both there and nothing else.
"""
import numpy as np
import pytest
import torch

from oracle import decide32
from oracle import field as OF
from oracle import occupancy as OO
from oracle import render as OR
from paper_2306_16541_gb300 import synth

from _util import nrmod, psnr

pytestmark = pytest.mark.gpu


def _shaped(seed, grid, res_last_std=0.02):
    s = synth.shaped_density(synth.subject(seed, with_ellipsoids=True, hash_scale=0.5, res_last_std=res_last_std))
    s["occ_grid"] = grid
    return s


def _canon_bounds(sigma, tau, grid, r):
    """(lo, hi): the dilated grids with every near-threshold cell off, then on."""
    sig = sigma.numpy()
    amb = np.abs(sig - tau) <= 1e-7 + 1e-4 * tau
    marked = sig > tau
    return OO.dilate(marked & ~amb, grid, r), OO.dilate(marked | amb, grid, r), int(amb.sum())


def _posed_bounds(canon, S, xf, grid, s_min):
    """(lo, hi) of the posed grid: a warped centre within a rounding band of a cell face may
    land in either cell, and S within a band of s_min may pass or fail."""
    S = S.numpy()
    _, u = OO.canonical_cell(xf, [-1, -1, -1], [1, 1, 1], grid)
    u = u.numpy()
    tol = 1e-3 * np.maximum(1.0, 1e-2 / np.maximum(S, 1e-12))
    base = np.floor(u)
    frac = u - base
    lo = np.ones(S.shape, bool)
    hi = np.zeros(S.shape, bool)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                d = np.array([dx, dy, dz])
                ok = np.ones(S.shape, bool)
                for k in range(3):
                    if d[k] == -1:
                        ok &= frac[:, k] < tol
                    elif d[k] == 1:
                        ok &= frac[:, k] > 1 - tol
                ci = np.clip(base + d, 0, grid - 1).astype(np.int64)
                bit = canon[(ci[:, 2] * grid + ci[:, 1]) * grid + ci[:, 0]]
                lo &= np.where(ok, bit, True)
                hi |= np.where(ok, bit, False)
    s_amb = np.abs(S - s_min) <= 1e-5
    lo &= (S >= s_min) & ~s_amb
    hi &= (S >= s_min) | s_amb
    return lo, hi


@pytest.mark.parametrize("grid,r,structured", [(32, 0, False), (32, 1, False), (64, 2, False), (32, 1, True)])
def test_canonical_refresh_matches_oracle(grid, r, structured):
    nr = nrmod()
    if structured:
        # an unshaped field (random MLP on a structured table): the threshold sits at the median
        s = synth.subject(44, hash_scale=0.5, hidden_layers=3)
        s["occ_grid"] = grid
        sigma = OO.canonical_sigma(OF.Params(s), grid)
        tau = float(sigma.median())
    else:
        s = _shaped(43, grid)
        tau = 1e-3
        sigma = OO.canonical_sigma(OF.Params(s), grid)
    lo, hi, n_amb = _canon_bounds(sigma, tau, grid, r)
    S = nr.Subject(s)
    try:
        S.refresh_occupancy(tau, r)
        got = OO.unpack(S.canonical_occupancy())
    finally:
        S.close()
    assert n_amb <= grid ** 3 // 200
    assert 0 < lo.sum() and hi.sum() < grid ** 3
    assert np.all(got >= lo) and np.all(got <= hi), (int((got < lo).sum()), int((got > hi).sum()))


@pytest.mark.parametrize("grid,s_min", [(32, 1e-3), (64, 0.3)])
def test_posed_grid_matches_oracle(grid, s_min):
    """A seeded canonical bitfield posed through the weight volume and a non-zero residual."""
    nr = nrmod()
    s = _shaped(45, grid)
    canon = np.random.default_rng(46).uniform(size=grid ** 3) < 0.3
    pose = synth.random_pose(np.random.default_rng(47))
    S = nr.Subject(s)
    try:
        S.set_canonical_occupancy(OO.pack(canon), s_min)
        S.set_pose(*pose)
        got = OO.unpack(S.occupancy())
        assert np.array_equal(OO.unpack(S.canonical_occupancy()), canon)
    finally:
        S.close()
    P = OF.Params(s)
    G_R, G_t, omega = OR.pose_inputs(s, *pose)
    Sw, xf = OO.posed_points(P, G_R, G_t, omega, grid)
    ref = OO.posed_grid(canon, Sw, xf, s["box_min"], s["box_max"], grid, s_min)
    lo, hi = _posed_bounds(canon, Sw, xf, grid, s_min)
    assert np.array_equal(lo, lo & ref) and np.array_equal(hi, hi | ref)
    assert int((lo != hi).sum()) <= grid ** 3 // 200
    assert ref.sum() > 0
    assert np.all(got >= lo) and np.all(got <= hi), (int((got < lo).sum()), int((got > hi).sum()))


def _ray_cells(s, cam, grid):
    py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    px, py = px.ravel(), py.ravel()
    o, d = decide32.ray_dirs32(cam, px, py)
    lo, hi, hit = decide32.clip32(o, d, cam.t_near, cam.t_far, s["box_min"], s["box_max"])
    x = decide32.sample_points32(o, d, lo, hi, cam.n_samples)
    return px, py, decide32.cell_of32(x, s["box_min"], s["box_max"], grid), hit


@pytest.mark.parametrize("mlp", ["f32", "bf16"])
def test_render_with_refreshed_grid_matches_oracle(mlp):
    nr = nrmod()
    grid, tau, r, s_min = 32, 1e-3, 1, 1e-3
    s = _shaped(48, grid)
    pose = synth.random_pose(np.random.default_rng(49))
    cam = synth.camera(40, 40, 50.0, (0.0, 0.0, 2.5), 32, 1.5, 3.5)
    S = nr.Subject(s)
    try:
        S.refresh_occupancy(tau, r, s_min)
        S.set_pose(*pose)
        img = S.render(cam, nr.make_opts(mlp, "f32", True, 0.0))
        torch.cuda.synchronize()
        img = img.cpu().numpy().reshape(-1, 4)
        got_posed = OO.unpack(S.occupancy())
    finally:
        S.close()
    P = OF.Params(s)
    canon, _ = OO.canonical_grid(P, grid, tau, r)
    G_R, G_t, omega = OR.pose_inputs(s, *pose)
    Sw, xf = OO.posed_points(P, G_R, G_t, omega, grid)
    posed = OO.posed_grid(canon, Sw, xf, s["box_min"], s["box_max"], grid, s_min)
    px, py, cells, _ = _ray_cells(s, cam, grid)
    differ = np.nonzero(got_posed != posed)[0]
    keep = ~np.isin(cells, differ).any(1)
    assert keep.mean() >= 0.9
    ref = OR.render_pixels(s, P, pose, cam, px, py, True, grid=grid, bits=OO.pack(posed)).numpy()
    if mlp == "f32":
        assert np.abs(img[keep] - ref[keep]).max() <= 1e-3
    else:
        assert psnr(img[keep], ref[keep]) >= 50.0
    assert ref[:, 3].max() > 0.5                       # the performer is in view


def test_skipping_with_the_grid_keeps_the_image():
    """Cells whose canonical density stays under the threshold carry almost no
    opacity, so skipping them changes no pixel by more than the skipped density
    can: the render with the refreshed grid equals the render without skipping."""
    nr = nrmod()
    s = _shaped(50, 128)
    pose = synth.random_pose(np.random.default_rng(51))
    cam = synth.camera(96, 96, 120.0, (0.0, 0.0, 2.5), 96, 1.5, 3.5)
    S = nr.Subject(s)
    try:
        S.set_pose(*pose)
        full = S.render(cam, nr.make_opts("f32", "f32", False, 0.0, profile=True))
        torch.cuda.synchronize()
        n_full = S.stage_times()["live_samples"]
        S.refresh_occupancy(1e-3, 1, 1e-3)
        skip = S.render(cam, nr.make_opts("f32", "f32", True, 0.0, profile=True))
        torch.cuda.synchronize()
        n_skip = S.stage_times()["live_samples"]
    finally:
        S.close()
    full, skip = full.cpu().numpy(), skip.cpu().numpy()
    assert full[..., 3].max() > 0.5
    assert np.abs(full - skip).max() <= 3e-3
    assert n_skip < 0.6 * n_full, (n_skip, n_full)


def test_parameter_change_reposes_the_grid():
    """The posed grid follows the parameters: with the bone weights zeroed every S is 0 and
    no cell survives the s_min test."""
    nr = nrmod()
    s = _shaped(52, 32)
    S = nr.Subject(s)
    try:
        S.refresh_occupancy(1e-3, 1, 1e-3)
        S.set_pose(*synth.random_pose(np.random.default_rng(53)))
        assert S.occupancy().any()
        S.param(nr.NR_PARAM_WVOL)[0].zero_()
        S.params_changed()
        assert not S.occupancy().any()
    finally:
        S.close()


def test_served_request_with_grid_occupancy_equals_render():
    nr = nrmod()
    s = _shaped(54, 64)
    sub = nr.Subject(s)
    sub.refresh_occupancy(1e-3, 1, 1e-3)
    srv = nr.Server(max_bytes=2 << 30, max_slots=2)
    try:
        srv.add_subject(sub)
        rng = np.random.default_rng(55)
        for k in range(3):
            aa, rt = synth.random_pose(rng)
            cam = synth.camera(48, 48, 60.0, synth.random_eye(rng), 32, 0.5, 4.5)
            opts = nr.make_opts(["f32", "bf16", "f32"][k], "f32", True, 1e-4)
            out = torch.full((48, 48, 4), float("nan"), device="cuda")
            srv.wait(srv.submit(srv.request(0, cam, aa, rt, opts, out)), 60000)
            sub.set_pose(aa, rt)
            alone = sub.render(cam, opts)
            torch.cuda.synchronize()
            assert torch.equal(out, alone)
    finally:
        srv.close()
        sub.close()
