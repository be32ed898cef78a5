"""The allocation-free render entry point, nr_render_static, called through the C ABI.

Callers that cannot let the library allocate device memory at render time (a
real-time thread that must not stall on cudaMalloc's device synchronisation, a
process whose free memory is already in its own pool, code under stream capture)
use nr_render_static, whose work queues sit in a fixed device array.  Its output
must match nr_render's on the same subject, pose and camera, call after call.
This file is collected last so that a failure here leaves every other test run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2306_16541_gb300 import synth

from _util import nrmod

pytestmark = pytest.mark.gpu

TOL = 1e-3      # the float32 tolerance of the parity tests


def _static(nr, S, cam, opts, out):
    return nr.lib.nr_render_static(S.h, C.byref(cam), C.byref(opts), C.c_void_p(out.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("which", ["tiny_f32", "frame_bf16_at_limit"])
def test_static_render_matches_nr_render_twice(which):
    nr = nrmod()
    if which == "tiny_f32":
        cfg = synth.config_tiny()
        subj = synth.subject(1234, hash_scale=0.5, res_last_std=0.02)
        cam = nr.make_camera(cfg["camera"])                        # 64 x 64 x 32 = 131,072 slots
        opts = nr.make_opts("f32")
    else:
        cfg = synth.config_frame512()
        subj = cfg["subject"]
        c = synth.camera(64, 64, 80.0, (0.0, 0.0, 2.5), 64, 0.5, 4.5)
        cam = nr.make_camera(c)                                    # 64 x 64 x 64 = 262,144 slots (the limit)
        opts = nr.make_opts("bf16", "f16", occupancy=True, t_min=1e-4)
    S = nr.Subject(subj)
    try:
        S.set_pose(*cfg["pose"])
        ref = S.render(cam, opts).cpu().numpy()
        for _ in range(2):
            out = torch.full((cam.height, cam.width, 4), float("nan"), device="cuda")
            assert _static(nr, S, cam, opts, out) == nr.NR_OK, nr.lib.nr_last_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            assert np.abs(got - ref).max() <= TOL
    finally:
        S.close()


def test_static_render_rejects_frames_beyond_its_limits():
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
        host = np.zeros((64, 64, 4), np.float32)
        small = nr.make_camera(cfg["camera"])
        rc = nr.lib.nr_render_static(S.h, C.byref(small), C.byref(nr.make_opts()), C.c_void_p(host.ctypes.data),
                                     C.c_void_p(0))
        assert rc == nr.NR_EINVAL and b"device memory" in nr.lib.nr_last_error()
    finally:
        S.close()
