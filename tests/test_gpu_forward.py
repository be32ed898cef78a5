"""Forward parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: the float32 path within 1e-3 max-abs RGBA of the oracle; the
bf16/f16 tensor-core tiers at PSNR >= 50 dB.  Integer decisions (which rays
hit the box, the posed occupancy bitfield, which samples are live) are taken
in float32 by both sides and must agree exactly.
"""
import numpy as np
import pytest
import torch

from oracle import decide32, fk
from oracle import field as OF
from paper_2306_16541_gb300 import synth

from _util import gpu_render, nrmod, oracle_render, psnr

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-3


@pytest.fixture(scope="module")
def tiny():
    return synth.config_tiny()


@pytest.fixture(scope="module")
def tiny_structured():
    cfg = synth.config_tiny()
    cfg["subject"] = synth.subject(1234, hash_scale=0.5, res_last_std=0.02)
    return cfg


@pytest.fixture(scope="module")
def frame():
    return synth.config_frame512()


def _small(cam, res, n_samples=None):
    c = synth.camera(res, res, 1.25 * res, (0.0, 0.0, 2.5), n_samples or cam.n_samples, cam.t_near, cam.t_far)
    c.R, c.t = cam.R, cam.t
    return c


def test_fk_matches_oracle(tiny):
    nr = nrmod()
    S = nr.Subject(tiny["subject"])
    try:
        S.set_pose(*tiny["pose"])
        G = S.pose_transforms()
    finally:
        S.close()
    s = tiny["subject"]
    ref = fk.bone_transforms_f32(s["parents"], s["rest_joints"], *tiny["pose"])
    assert np.abs(G - ref).max() <= 1e-6


def test_posed_bitfield_bit_exact(frame):
    nr = nrmod()
    s = frame["subject"]
    G32 = fk.bone_transforms_f32(s["parents"], s["rest_joints"], *frame["pose"])
    S = nr.Subject(s)
    try:
        S.set_pose(G32, matrices=True)
        bits = S.occupancy()
    finally:
        S.close()
    ref = decide32.posed_bitfield32(G32, s["ellipsoids"], s["box_min"], s["box_max"], 128)
    assert np.array_equal(bits, ref), int(np.count_nonzero(bits != ref))
    frac = np.unpackbits(bits.view(np.uint8)).mean()
    assert 0.1 < frac < 0.3


def test_query_matches_oracle(tiny_structured):
    nr = nrmod()
    cfg = tiny_structured
    s = cfg["subject"]
    x = np.random.default_rng(3).uniform(-0.9, 0.9, size=(4099, 3)).astype(np.float32)
    S = nr.Subject(s)
    try:
        S.set_pose(*cfg["pose"])
        out = S.query(torch.from_numpy(x).cuda()).cpu().numpy()
    finally:
        S.close()
    P = OF.Params(s)
    R, t = fk.bone_transforms(s["parents"], s["rest_joints"], *cfg["pose"])
    ref = OF.field(torch.from_numpy(x.astype(np.float64)), P, torch.from_numpy(R), torch.from_numpy(t),
                   torch.from_numpy(cfg["pose"][0].astype(np.float64)).reshape(-1))
    S_ref = ref["S"].numpy()
    assert np.abs(out[:, 3] - S_ref).max() < 1e-5
    m = S_ref > 1e-2                                   # x_skel is well conditioned there
    assert m.sum() > 500
    assert np.abs(out[m, 0:3] - ref["x_skel"].numpy()[m]).max() < 1e-4
    assert np.abs(out[m, 4:7] - ref["x_final"].numpy()[m]).max() < 1e-4
    inside = ref["inside"].numpy()
    assert np.array_equal(out[m, 7] > 0.5, inside[m])
    mi = m & inside
    assert np.abs(out[mi, 8:11] - ref["rgb"].numpy()[mi]).max() < 1e-3
    assert np.abs(out[mi, 11] - ref["sigma"].numpy()[mi]).max() < 1e-3


@pytest.mark.parametrize("structured", [False, True])
def test_render_tiny_f32(tiny, tiny_structured, structured):
    cfg = tiny_structured if structured else tiny
    got = gpu_render(cfg["subject"], cfg["pose"], cfg["camera"], False)
    ref = oracle_render(cfg["subject"], cfg["pose"], cfg["camera"], False).reshape(got.shape)
    err = np.abs(got - ref).max()
    assert err <= TOL_F32, err
    assert ref[..., 3].max() > 0.1


def test_render_host_buffer_equals_device(tiny_structured):
    cfg = tiny_structured
    a = gpu_render(cfg["subject"], cfg["pose"], cfg["camera"], False)
    b = gpu_render(cfg["subject"], cfg["pose"], cfg["camera"], False, host=True)
    assert np.array_equal(a, b)


def test_render_frame_field_with_occupancy(frame):
    """The 512x512 workload's field (16 levels of 2^19 f16 entries, 64^3 volume,
    3 hidden layers, occupancy) rendered at 64x64, every pixel against the oracle."""
    cam = _small(frame["camera"], 64)
    got = gpu_render(frame["subject"], frame["pose"], cam, True, feat="f16")
    ref = oracle_render(frame["subject"], frame["pose"], cam, True).reshape(got.shape)
    err = np.abs(got - ref).max()
    assert err <= TOL_F32, err


def test_render_frame_full_size_sampled(frame):
    """512x512, 128 samples, occupancy, as the bench launches it; 1500 sampled pixels."""
    cam = frame["camera"]
    got = gpu_render(frame["subject"], frame["pose"], cam, True, feat="f16")
    rng = np.random.default_rng(0)
    px = rng.integers(0, cam.width, 1500)
    py = rng.integers(0, cam.height, 1500)
    ref = oracle_render(frame["subject"], frame["pose"], cam, True, px, py)
    err = np.abs(got[py, px] - ref).max()
    assert err <= TOL_F32, err


def test_early_termination_bound(tiny_structured):
    cfg = dict(tiny_structured)
    s = synth.subject(77, hash_scale=0.5)
    # dense field: large positive sigma bias so rays terminate early
    s["mlp_layers"][-1][1][3] = 40.0
    s["mlp_params"] = synth.pack_layers(s["mlp_layers"])
    full = gpu_render(s, cfg["pose"], cfg["camera"], False, t_min=0.0)
    ert = gpu_render(s, cfg["pose"], cfg["camera"], False, t_min=1e-4)
    assert (1 - full[..., 3]).min() < 1e-4                # some rays do terminate
    assert np.abs(full - ert).max() <= 1e-4


def test_rays_missing_the_box_get_background(tiny):
    cfg = tiny
    cam = synth.camera(16, 8, 20.0, (0.0, 0.0, 2.5), 8, 1.5, 3.5, bg=(0.25, 0.5, 0.75))
    R, t = synth.look_at((0.0, 0.0, 2.5), target=(0.0, 5.0, 2.5), up=(0.0, 0.0, 1.0))
    cam.R, cam.t = R, t                                   # looking straight up, away from the box
    got = gpu_render(cfg["subject"], cfg["pose"], cam, False)
    assert np.allclose(got[..., :3], [0.25, 0.5, 0.75]) and (got[..., 3] == 0).all()


@pytest.mark.parametrize("res,S", [(1, 1), (3, 7), (17, 33)])
def test_ragged_sizes(tiny_structured, res, S):
    cfg = tiny_structured
    cam = _small(cfg["camera"], res, S)
    got = gpu_render(cfg["subject"], cfg["pose"], cam, False)
    ref = oracle_render(cfg["subject"], cfg["pose"], cam, False).reshape(got.shape)
    assert np.abs(got - ref).max() <= TOL_F32


@pytest.mark.parametrize("mlp", ["bf16", "f16"])
@pytest.mark.parametrize("feat", ["f32", "f16"])
def test_tensor_core_tiers_psnr(tiny_structured, mlp, feat):
    """Reduced-precision tiers against the oracle: PSNR >= 50 dB (and reported max-abs)."""
    cfg = tiny_structured
    s = dict(cfg["subject"])
    # f16 storage of the table: the tier reads entries rounded to f16
    got = gpu_render(s, cfg["pose"], cfg["camera"], False, mlp=mlp, feat=feat)
    ref = oracle_render(s, cfg["pose"], cfg["camera"], False).reshape(got.shape)
    p = psnr(got, ref)
    assert p >= 50.0, (p, float(np.abs(got - ref).max()))


@pytest.mark.parametrize("mlp", ["bf16", "f16"])
def test_tensor_core_tier_frame_field(frame, mlp):
    cam = _small(frame["camera"], 64)
    got = gpu_render(frame["subject"], frame["pose"], cam, True, mlp=mlp, feat="f16")
    ref = oracle_render(frame["subject"], frame["pose"], cam, True).reshape(got.shape)
    assert psnr(got, ref) >= 50.0


def test_tensor_core_query_matches_f32(tiny_structured):
    """Per-sample outputs of the bf16 tier against the float32 tier on the same points."""
    nr = nrmod()
    cfg = tiny_structured
    x = torch.from_numpy(np.random.default_rng(5).uniform(-0.9, 0.9, size=(1000, 3)).astype(np.float32)).cuda()
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        a = S.query(x, nr.make_opts("f32")).cpu().numpy()
        b = S.query(x, nr.make_opts("bf16")).cpu().numpy()
    finally:
        S.close()
    assert np.array_equal(a[:, :4], b[:, :4])            # the warp is float32 in both tiers
    m = a[:, 3] > 1e-2
    assert np.abs(a[m, 4:7] - b[m, 4:7]).max() < 2e-3    # x_final through the bf16 residual MLP
    assert np.abs(a[m, 8:11] - b[m, 8:11]).max() < 3e-2


FP8_PSNR_DB = 50.0   # the reduced-precision bar; e4m3 keeps 3 mantissa bits (elements off by up to 1/16)


@pytest.mark.parametrize("path", ["pipeline", "mma_sync"])
@pytest.mark.parametrize("which", ["tiny_structured", "frame"])
def test_fp8_tier_psnr(tiny_structured, frame, which, path):
    """FP8 E4M3 MLPs (per-matrix weight scales, calibrated static activation scales) against
    the oracle, on the tcgen05 pipeline (kind::f8f6f4, the default) and on mma.sync; the measured
    PSNR is printed for the precision table."""
    if which == "frame":
        cfg, cam, occ = frame, _small(frame["camera"], 64), True
    else:
        cfg, cam, occ = tiny_structured, tiny_structured["camera"], False
    got = gpu_render(cfg["subject"], cfg["pose"], cam, occ, mlp="fp8", feat="f16" if occ else "f32",
                     mma_sync=(path == "mma_sync"))
    ref = oracle_render(cfg["subject"], cfg["pose"], cam, occ).reshape(got.shape)
    p = psnr(got, ref)
    print(f"fp8 {which} {path}: PSNR {p:.2f} dB, max abs {np.abs(got - ref).max():.3e}")
    assert got[..., 3].max() > 0.1
    assert p >= FP8_PSNR_DB


@pytest.mark.parametrize("path", ["pipeline", "mma_sync"])
def test_fp8_is_batch_independent(tiny_structured, path):
    """Static scales: a point's fp8 result is the same whatever else is evaluated with it."""
    nr = nrmod()
    cfg = tiny_structured
    x = torch.from_numpy(np.random.default_rng(8).uniform(-0.9, 0.9, size=(2000, 3)).astype(np.float32)).cuda()
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        o = nr.make_opts("fp8", mma_sync=(path == "mma_sync"))
        full = S.query(x, o)
        part = S.query(x[:333].contiguous(), o)
        torch.cuda.synchronize()
        assert torch.equal(full[:333], part)
    finally:
        S.close()


def _render_opts(mlp, feat, occ, tcgen05):
    nr = nrmod()
    return nr.make_opts(mlp, feat, occ, 0.0, tcgen05=tcgen05)


@pytest.mark.parametrize("mlp", ["bf16", "f16"])
def test_tcgen05_path_psnr_and_agreement(tiny_structured, frame, mlp):
    """bf16/f16 MLPs on tcgen05.mma with TMEM accumulators: PSNR >= 50 dB against the oracle,
    and close to the warp-level mma.sync path (same operand rounding, other summation order)."""
    nr = nrmod()
    for cfg, cam, occ, feat in ((tiny_structured, tiny_structured["camera"], False, "f32"),
                                (frame, _small(frame["camera"], 64), True, "f16")):
        S = nr.Subject(cfg["subject"])
        try:
            S.set_pose(*cfg["pose"])
            a = S.render(cam, _render_opts(mlp, feat, occ, True)).cpu().numpy()
            b = S.render(cam, _render_opts(mlp, feat, occ, False)).cpu().numpy()
        finally:
            S.close()
        ref = oracle_render(cfg["subject"], cfg["pose"], cam, occ).reshape(a.shape)
        assert psnr(a, ref) >= 50.0, psnr(a, ref)
        assert np.abs(a - b).max() <= 2e-2 and psnr(a, b) >= 55.0, (np.abs(a - b).max(), psnr(a, b))


@pytest.mark.parametrize("mlp", ["bf16", "f16"])
def test_two_tile_path_equals_default(frame, mlp):
    """NR_RENDER_MMA2 (two 16-row tiles per weight-fragment read, each layer taken in
    output-column order) issues the same MMAs on every accumulator, in the same order, as
    the one-tile mma.sync path: images and query rows are bitwise equal, a ragged tail included."""
    nr = nrmod()
    cam = _small(frame["camera"], 96)
    x = torch.from_numpy(np.random.default_rng(10).uniform(-0.9, 0.9, size=(1001, 3)).astype(np.float32)).cuda()
    S = nr.Subject(frame["subject"])
    try:
        S.set_pose(*frame["pose"])
        a = S.render(cam, nr.make_opts(mlp, "f16", True, 1e-4, mma_sync=True))
        b = S.render(cam, nr.make_opts(mlp, "f16", True, 1e-4, mma2=True))
        qa = S.query(x, nr.make_opts(mlp, "f16", mma_sync=True))
        qb = S.query(x, nr.make_opts(mlp, "f16", mma2=True))
        torch.cuda.synchronize()
    finally:
        S.close()
    assert a[..., 3].max().item() > 0.1
    assert torch.equal(a, b)
    assert torch.equal(qa, qb)


def test_tcgen05_query_ragged_tail(tiny_structured):
    """A point count that leaves a partial 128-sample tile; rows beyond n are never written."""
    nr = nrmod()
    cfg = tiny_structured
    x = torch.from_numpy(np.random.default_rng(9).uniform(-0.9, 0.9, size=(1000, 3)).astype(np.float32)).cuda()
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        out = torch.full((1003, nr.NR_QUERY_STRIDE), 7.0, device="cuda")
        nr.nr_query(S.h, x[:1000].contiguous(), nr.make_opts("bf16", tcgen05=True), out)
        ref = S.query(x, nr.make_opts("bf16"))
        torch.cuda.synchronize()
    finally:
        S.close()
    assert (out[1000:] == 7.0).all()
    a, b = out[:1000].cpu().numpy(), ref.cpu().numpy()
    assert np.array_equal(a[:, :4], b[:, :4])
    assert np.abs(a[:, 8:12] - b[:, 8:12]).max() < 2e-2


def test_bench_configuration_sampled_against_oracle(frame):
    """The frame exactly as bench.py times it (512x512, 128 samples, occupancy, f16 table,
    bf16 MLPs on the default path, ERT at 1e-4): 2000 sampled pixels against the oracle.
    ERT changes a pixel by at most T_min, inside the PSNR budget."""
    nr = nrmod()
    cam = frame["camera"]
    S = nr.Subject(frame["subject"])
    try:
        S.set_pose(*frame["pose"])
        img = S.render(cam, nr.make_opts("bf16", "f16", True, 1e-4)).cpu().numpy()
    finally:
        S.close()
    rng = np.random.default_rng(5)
    px = rng.integers(0, cam.width, 2000)
    py = rng.integers(0, cam.height, 2000)
    ref = oracle_render(frame["subject"], frame["pose"], cam, True, px, py)
    got = img[py, px]
    assert psnr(got, ref) >= 50.0
    assert np.abs(got - ref).max() <= 1e-2


def test_round_based_termination_saves_work_and_matches_single_pass(tiny_structured):
    """Early termination in rounds: an opaque performer evaluates fewer samples than without
    termination, and the image equals the single-pass compositor that stops at the same T_min
    (nr_render_static composites every queued sample in one pass)."""
    import ctypes as C
    nr = nrmod()
    cfg = tiny_structured
    s = synth.subject(78, hash_scale=0.5)
    s["mlp_layers"][-1][1][3] = 40.0                      # opaque: rays terminate after a few samples
    s["mlp_params"] = synth.pack_layers(s["mlp_layers"])
    s["wvol"] = np.full_like(s["wvol"], 1.0 / 25.0)       # S = 24/25 everywhere in the box
    c = synth.camera(64, 64, 80.0, (0.0, 0.0, 2.5), 64, 1.5, 3.5)
    c.R, c.t = cfg["camera"].R, cfg["camera"].t
    cam = nr.make_camera(c)                               # 64 samples: four rounds of 16
    S = nr.Subject(s)
    try:
        S.set_pose(*cfg["pose"])
        on = nr.make_opts("f32", "f32", False, 1e-4, profile=True)
        off = nr.make_opts("f32", "f32", False, 0.0, profile=True)
        a = S.render(cam, on).clone()
        live_on = S.stage_times()["live_samples"]
        S.render(cam, off)
        live_off = S.stage_times()["live_samples"]
        b = torch.empty_like(a)
        rc = nr.lib.nr_render_static(S.h, C.byref(cam), C.byref(nr.make_opts("f32", "f32", False, 1e-4)),
                                     C.c_void_p(b.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == nr.NR_OK
        torch.cuda.synchronize()
    finally:
        S.close()
    assert live_on < 0.4 * live_off, (live_on, live_off)
    assert torch.equal(a, b)


@pytest.mark.parametrize("mlp", ["f32", "bf16"])
def test_bone_skipping_changes_nothing_visible(mlp):
    """Rendering skips bone channels whose support box misses the candidate point (their
    weights are <= 1e-7 there); against evaluating all 24 channels the image moves by no
    more than those weights can move it."""
    nr = nrmod()
    cfg = synth.config_frame512(structured=True)
    cam = synth.camera(96, 96, 120.0, (0.0, 0.0, 2.5), 64, 0.5, 4.5)
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        skip = S.render(cam, nr.make_opts(mlp, "f16", True, 1e-4)).cpu().numpy()
        full = S.render(cam, nr.make_opts(mlp, "f16", True, 1e-4, all_bones=True)).cpu().numpy()
    finally:
        S.close()
    assert full[..., 3].max() > 0.2
    assert np.abs(skip - full).max() <= 1e-4, np.abs(skip - full).max()


def test_f32_tensor_core_tier(tiny_structured, frame):
    """NR_RENDER_F32_TC: both MLPs as warp-level tensor-core layers with three TF32 products
    per step.  Within the float32 bar of the oracle (max abs <= 1e-3) on the tiny workload and
    on the frame workload with occupancy, within 1e-5 of the CUDA-core float32 path, query
    rows likewise (the warp's gathers are the same code: bitwise), and refused by
    nr_render_static, which allocates nothing."""
    import ctypes as C
    nr = nrmod()
    for cfg, cam, occ in ((tiny_structured, tiny_structured["camera"], False),
                          (frame, _small(frame["camera"], 64), True)):
        S = nr.Subject(cfg["subject"])
        try:
            S.set_pose(*cfg["pose"])
            tc = S.render(cam, nr.make_opts("f32", "f32", occ, 0.0, f32_tc=True)).cpu().numpy()
            fm = S.render(cam, nr.make_opts("f32", "f32", occ, 0.0)).cpu().numpy()
        finally:
            S.close()
        ref = oracle_render(cfg["subject"], cfg["pose"], cam, occ).reshape(tc.shape)
        assert ref[..., 3].max() > 0.1
        assert np.abs(tc - ref).max() <= 1e-3, np.abs(tc - ref).max()
        assert np.abs(tc - fm).max() <= 1e-5, np.abs(tc - fm).max()
    x = torch.from_numpy(np.random.default_rng(12).uniform(-0.9, 0.9, size=(1001, 3)).astype(np.float32)).cuda()
    S = nr.Subject(frame["subject"])
    try:
        S.set_pose(*frame["pose"])
        qa = S.query(x, nr.make_opts("f32", "f32", f32_tc=True)).cpu().numpy()
        qb = S.query(x, nr.make_opts("f32", "f32")).cpu().numpy()
        out = torch.empty(32, 32, 4, device="cuda")
        cam = nr.make_camera(_small(frame["camera"], 32))
        rc = nr.lib.nr_render_static(S.h, C.byref(cam), C.byref(nr.make_opts("f32", "f32", f32_tc=True)),
                                     C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
    finally:
        S.close()
    assert rc == nr.NR_EUNSUPPORTED
    assert np.array_equal(qa[:, :4], qb[:, :4])
    assert np.abs(qa[:, 4:] - qb[:, 4:]).max() <= 1e-4 * max(1.0, np.abs(qb[:, 4:]).max())


def test_pose_set_on_one_stream_reaches_renders_on_another(frame):
    """nr_set_pose queues its device work and returns; a render or a transform read issued on
    another stream right after it, with no host synchronisation between, must see that pose:
    each image equals the one rendered with pose and render on the same stream, bit for bit,
    and the transforms equal the oracle's forward kinematics.  (The other direction, a new pose
    after a render still running on another stream, is the caller's to order.)"""
    nr = nrmod()
    cam = nr.make_camera(_small(frame["camera"], 64))
    opts = nr.make_opts("bf16", "f16", True, 1e-4)
    rng = np.random.default_rng(77)
    poses = [synth.random_pose(rng) for _ in range(6)]
    S = nr.Subject(frame["subject"])
    try:
        ref = []
        for p in poses:
            S.set_pose(*p)
            ref.append(S.render(cam, opts).cpu().numpy())
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        outs = [torch.empty(cam.height, cam.width, 4, device="cuda") for _ in range(3 * len(poses))]
        torch.cuda.synchronize()
        for i, o in enumerate(outs):
            S.set_pose(*poses[i % len(poses)], stream=s1)
            S.render(cam, opts, o, stream=s2)
            s1.wait_stream(s2)      # the caller orders the next pose after a render that reads this one
        torch.cuda.synchronize()
        for i, o in enumerate(outs):
            assert np.array_equal(o.cpu().numpy(), ref[i % len(poses)]), i
        s = frame["subject"]
        for p in poses[:2]:
            S.set_pose(*p, stream=s1)
            G = S.pose_transforms()                 # legacy default stream, synchronous read
            assert np.abs(G - fk.bone_transforms_f32(s["parents"], s["rest_joints"], *p)).max() <= 1e-6
    finally:
        S.close()
