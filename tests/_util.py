"""Helpers shared by the GPU tests: build the library, run the oracle, compare."""
import functools

import numpy as np
import torch


@functools.lru_cache(maxsize=None)
def nrmod():
    from paper_2306_16541_gb300 import build
    build.build()
    from paper_2306_16541_gb300 import nr
    return nr


def psnr(a, b, peak=1.0):
    mse = float(((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2).mean())
    return float("inf") if mse == 0 else 10 * np.log10(peak * peak / mse)


def gpu_render(subj, pose, cam, occupancy, mlp="f32", feat="f32", t_min=0.0, host=False, matrices=None, **flags):
    nr = nrmod()
    S = nr.Subject(subj)
    try:
        if matrices is not None:
            S.set_pose(matrices, matrices=True)
        else:
            S.set_pose(*pose)
        opts = nr.make_opts(mlp, feat, occupancy, t_min, **flags)
        if host:
            out = np.zeros((cam.height, cam.width, 4), np.float32)
            S.render(cam, opts, out)
            return out
        out = S.render(cam, opts)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        S.close()


def oracle_render(subj, pose, cam, occupancy, px=None, py=None):
    from oracle import field as OF
    from oracle import render as OR
    P = OF.Params(subj)
    if px is None:
        py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
        px, py = px.ravel(), py.ravel()
    return OR.render_pixels(subj, P, pose, cam, px, py, occupancy).numpy()
