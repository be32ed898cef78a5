"""The warp-specialised tcgen05 field pipeline (the bf16/f16 default) through the C ABI.

Both MLPs run as M = 128 tcgen05 MMAs with A read from tensor memory; the
operands are rounded as on the warp-level mma.sync path (NR_RENDER_MMA_SYNC),
the hidden biases are carried as bf16/f16 hi + lo pairs inside the products and
the summation order differs: images are held to PSNR >= 50 dB against the FP64
oracle (the reduced-precision bar) and close to the mma.sync path.  The gathers
compute the same float32 values in the same order, so the warp outputs (x_skel,
S) of a query are bitwise those of the mma.sync path.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2306_16541_gb300 import synth

from _util import nrmod, oracle_render, psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_structured():
    cfg = synth.config_tiny()
    cfg["subject"] = synth.subject(1234, hash_scale=0.5, res_last_std=0.02)
    return cfg


@pytest.fixture(scope="module")
def frame_structured():
    return synth.config_frame512(structured=True)


def _small(cam, res):
    c = synth.camera(res, res, 1.25 * res, (0.0, 0.0, 2.5), cam.n_samples, cam.t_near, cam.t_far)
    c.R, c.t = cam.R, cam.t
    return c


def _pair(nr, cfg, cam, mlp, feat, occ, t_min=0.0):
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        a = S.render(cam, nr.make_opts(mlp, feat, occ, t_min)).cpu().numpy()
        b = S.render(cam, nr.make_opts(mlp, feat, occ, t_min, mma_sync=True)).cpu().numpy()
    finally:
        S.close()
    return a, b


@pytest.mark.parametrize("mlp", ["bf16", "f16"])
def test_ws_psnr_against_oracle_and_agreement(tiny_structured, frame_structured, mlp):
    nr = nrmod()
    cases = ((tiny_structured, tiny_structured["camera"], False, "f32"),
             (frame_structured, _small(frame_structured["camera"], 64), True, "f16"))
    for cfg, cam, occ, feat in cases:
        a, b = _pair(nr, cfg, cam, mlp, feat, occ)
        ref = oracle_render(cfg["subject"], cfg["pose"], cam, occ).reshape(a.shape)
        assert a[..., 3].max() > 0.1
        assert psnr(a, ref) >= 50.0, psnr(a, ref)
        assert np.abs(a - b).max() <= 2e-2 and psnr(a, b) >= 55.0, (np.abs(a - b).max(), psnr(a, b))


@pytest.mark.parametrize("mlp", ["bf16", "fp8"])
def test_ws_without_residual_and_two_hidden_layers(tiny_structured, mlp):
    # the tiny workload's canonical MLP has two hidden layers; with MLP_res off the pipeline runs
    # only the canonical layers (another layer count per tile, and for fp8 another scale table)
    nr = nrmod()
    cfg = dict(tiny_structured)
    cfg["subject"] = dict(cfg["subject"], res_enabled=0)
    cam = cfg["camera"]
    a, b = _pair(nr, cfg, cam, mlp, "f32", False)
    ref = oracle_render(cfg["subject"], cfg["pose"], cam, False).reshape(a.shape)
    assert psnr(a, ref) >= 50.0, psnr(a, ref)
    assert psnr(a, b) >= (55.0 if mlp == "bf16" else 45.0), psnr(a, b)


def test_ws_query_ragged_tail_and_warp_outputs(tiny_structured):
    """1000 points leave a partial 128-row tile; rows beyond n are never written; the inverse-LBS
    outputs are the mma.sync path's bit for bit, the colours and density agree closely."""
    nr = nrmod()
    cfg = tiny_structured
    x = torch.from_numpy(np.random.default_rng(9).uniform(-0.9, 0.9, size=(1000, 3)).astype(np.float32)).cuda()
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        out = torch.full((1003, nr.NR_QUERY_STRIDE), 7.0, device="cuda")
        nr.nr_query(S.h, x, nr.make_opts("bf16"), out)
        ref = S.query(x, nr.make_opts("bf16", mma_sync=True))
        torch.cuda.synchronize()
    finally:
        S.close()
    assert (out[1000:] == 7.0).all()
    a, b = out[:1000].cpu().numpy(), ref.cpu().numpy()
    assert np.array_equal(a[:, :4], b[:, :4])
    assert np.abs(a[:, 4:7] - b[:, 4:7]).max() < 2e-3        # x_final: x_skel + a bf16 MLP_res
    assert np.abs(a[:, 8:12] - b[:, 8:12]).max() < 2e-2


@pytest.mark.parametrize("n", [1, 127, 128, 129, 152 * 4 * 128 + 5])
def test_ws_tile_counts(tiny_structured, n):
    """Sample counts below one tile, at a tile boundary, and beyond one tile per group of every
    block (several tiles per group): each row equals the single-point query of the same path."""
    nr = nrmod()
    cfg = tiny_structured
    g = np.random.default_rng(n)
    x = torch.from_numpy(g.uniform(-0.9, 0.9, size=(n, 3)).astype(np.float32)).cuda()
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        full = S.query(x, nr.make_opts("bf16"))
        pick = np.unique(g.integers(0, n, 8))
        singles = [S.query(x[i:i + 1].contiguous(), nr.make_opts("bf16")) for i in pick]
        torch.cuda.synchronize()
    finally:
        S.close()
    for i, row in zip(pick, singles):
        assert torch.equal(full[i], row[0])


def test_ws_full_frame_against_oracle(frame_structured):
    """The bench's frame (512 x 512 x 128, occupancy, f16 table, ERT 1e-4) on a textured field in
    bf16 through the pipeline: 2000 sampled pixels against the oracle."""
    nr = nrmod()
    cfg = frame_structured
    cam = cfg["camera"]
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        img = S.render(cam, nr.make_opts("bf16", "f16", True, 1e-4)).cpu().numpy()
    finally:
        S.close()
    rng = np.random.default_rng(5)
    px = rng.integers(0, cam.width, 2000)
    py = rng.integers(0, cam.height, 2000)
    ref = oracle_render(cfg["subject"], cfg["pose"], cam, True, px, py)
    got = img[py, px]
    err = np.abs(got - ref)
    print(f"ws bf16 structured 512^2: PSNR {psnr(got, ref):.1f} dB, max {err.max():.2e}, "
          f"p99 {np.percentile(err.max(1), 99):.2e}")
    assert psnr(got, ref) >= 50.0


def test_ws_error_word_makes_the_call_report_a_timeout(tiny_structured):
    """The word the pipeline sets when a bounded wait gives up is read back by the call: a word
    written from the host before a render makes that render return NR_ETIMEOUT with a message,
    and the call after it succeeds again (the word is cleared)."""
    nr = nrmod()
    cfg = tiny_structured
    cam = cfg["camera"]
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        ptr = C.c_void_p()
        opts = nr.make_opts("bf16")
        S.render(cam, opts)
        assert nr.lib.nr_field_error_word(S.h, C.byref(ptr)) == nr.NR_OK
        word = torch.as_tensor(_U32(ptr.value), device="cuda")
        assert int(word.item()) == 0
        word.fill_(1)
        torch.cuda.synchronize()
        out = torch.empty(cam.height, cam.width, 4, device="cuda")
        rc = nr.lib.nr_render(S.h, C.byref(nr.make_camera(cam)), C.byref(opts), C.c_void_p(out.data_ptr()),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == nr.NR_ETIMEOUT
        assert b"bounded wait" in nr.lib.nr_last_error()
        assert int(word.item()) == 0
        S.render(cam, opts)
        torch.cuda.synchronize()
    finally:
        S.close()


class _U32:
    def __init__(self, ptr):
        self.__cuda_array_interface__ = {"shape": (1,), "typestr": "<i4", "data": (ptr, False), "version": 3,
                                         "strides": None}


def test_profiled_render_counts_the_bone_channels_read(frame_structured):
    """A profiled render reports how many weight-volume channels the pipeline read per live
    sample: at least one (a sample on the body), fewer than the 24 bones (support skipping),
    and none reported by the mma.sync path, which does not count."""
    nr = nrmod()
    cfg = frame_structured
    cam = _small(cfg["camera"], 96)
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        S.render(cam, nr.make_opts("bf16", "f16", True, 1e-4, profile=True))
        st = S.stage_times()
        S.render(cam, nr.make_opts("bf16", "f16", True, 1e-4, profile=True, mma_sync=True))
        st_sync = S.stage_times()
    finally:
        S.close()
    assert st["live_samples"] == st_sync["live_samples"] > 0
    assert 1.0 <= st["bones_read_per_sample"] < 24.0, st
    assert st_sync["bones_read_per_sample"] == 0.0
