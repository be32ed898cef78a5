"""The allocation-free render entry point, nr_render_static, called through the C ABI.

Callers that cannot let the library allocate device memory at render time (a
real-time thread that must not stall on cudaMalloc's device synchronisation, a
process whose free memory is already in its own pool) use nr_render_static,
whose work queues sit in a fixed device array.  It runs the same kernels in the
same order as nr_render, so its image must equal nr_render's bit for bit, call
after call, and match the FP64 oracle like any render; free device memory must
not move across a call.  This file is collected last so that a failure here
leaves every other test run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2306_16541_gb300 import synth

from _util import nrmod, oracle_render, psnr

pytestmark = pytest.mark.gpu

TOL = 1e-3      # the float32 tolerance of the parity tests


def _static(nr, S, cam, opts, out):
    return nr.lib.nr_render_static(S.h, C.byref(cam), C.byref(opts), C.c_void_p(out.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _case(nr, which):
    if which == "tiny_f32":
        cfg = synth.config_tiny()
        subj = synth.subject(1234, hash_scale=0.5, res_last_std=0.02)
        c = cfg["camera"]                                          # 64 x 64 x 32 = 131,072 slots
        return subj, cfg["pose"], c, [nr.make_opts("f32")], False
    cfg = synth.config_frame512(structured=True)
    c = synth.camera(64, 64, 80.0, (0.0, 0.0, 2.5), 64, 0.5, 4.5)  # 64 x 64 x 64 = 262,144 slots (the limit)
    opts = [nr.make_opts("bf16", "f16", occupancy=True, t_min=1e-4),
            nr.make_opts("bf16", "f16", occupancy=True, t_min=1e-4, mma2=True),
            nr.make_opts("bf16", "f16", occupancy=True, t_min=1e-4, mma_sync=True)]
    return cfg["subject"], cfg["pose"], c, opts, True


@pytest.mark.parametrize("which", ["tiny_f32", "frame_bf16_at_limit"])
def test_static_render_matches_nr_render_and_the_oracle(which):
    nr = nrmod()
    subj, pose, c, opts_list, occ = _case(nr, which)
    cam = nr.make_camera(c)
    S = nr.Subject(subj)
    try:
        S.set_pose(*pose)
        outs = [torch.full((cam.height, cam.width, 4), float("nan"), device="cuda") for _ in range(2)]
        for opts in opts_list:
            # a fresh subject's first render is the static one; then the same call again, with
            # free device memory read on both sides of the second call
            assert _static(nr, S, cam, opts, outs[0]) == nr.NR_OK, nr.lib.nr_last_error()
            torch.cuda.synchronize()
            free0, _ = torch.cuda.mem_get_info()
            assert _static(nr, S, cam, opts, outs[1]) == nr.NR_OK, nr.lib.nr_last_error()
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            assert free1 == free0
            ref = S.render(cam, opts).cpu().numpy()
            for o in outs:
                got = o.cpu().numpy()
                assert np.isfinite(got).all()
                assert np.array_equal(got, ref)
        oracle = oracle_render(subj, pose, c, occ).reshape(ref.shape)
        if which == "tiny_f32":
            assert np.abs(ref - oracle).max() <= TOL
        else:
            assert ref[..., 3].max() > 0.1
            assert psnr(ref, oracle) >= 50.0, psnr(ref, oracle)
    finally:
        S.close()


def test_static_render_rejects_frames_beyond_its_limits_and_unsupported_flags():
    nr = nrmod()
    cfg = synth.config_tiny()
    S = nr.Subject(cfg["subject"])
    try:
        S.set_pose(*cfg["pose"])
        out = torch.zeros(512, 512, 4, device="cuda")
        big = nr.make_camera(synth.camera(512, 512, 640.0, (0.0, 0.0, 2.5), 1, 1.5, 3.5))
        assert _static(nr, S, big, nr.make_opts(), out) == nr.NR_EINVAL
        assert b"rays exceed the static limit" in nr.lib.nr_last_error()
        deep = nr.make_camera(synth.camera(64, 64, 80.0, (0.0, 0.0, 2.5), 128, 1.5, 3.5))
        assert _static(nr, S, deep, nr.make_opts(), out) == nr.NR_EINVAL
        assert b"sample slots exceed the static limit" in nr.lib.nr_last_error()
        small = nr.make_camera(cfg["camera"])
        assert _static(nr, S, small, nr.make_opts("f32", f32_tc=True), out) == nr.NR_EUNSUPPORTED
        assert _static(nr, S, small, nr.make_opts("bf16", profile=True), out) == nr.NR_EUNSUPPORTED
        assert _static(nr, S, small, nr.make_opts("fp8"), out) == nr.NR_EINVAL
        host = np.zeros((64, 64, 4), np.float32)
        rc = nr.lib.nr_render_static(S.h, C.byref(small), C.byref(nr.make_opts()), C.c_void_p(host.ctypes.data),
                                     C.c_void_p(0))
        assert rc == nr.NR_EINVAL and b"device memory" in nr.lib.nr_last_error()
    finally:
        S.close()
