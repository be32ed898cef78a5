"""The library's hand-written backward behind torch.autograd (nr.RenderFn): gradients of a
loss written in torch equal the library's fused MSE step, agree with the FP64 oracle for a
loss the library does not know (L1), and torch.optim steps the library's own parameters."""
import numpy as np
import pytest
import torch

from oracle import field as OF
from oracle import render as OR
from paper_2306_16541_gb300 import synth

from _util import nrmod

pytestmark = pytest.mark.gpu


def u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _linear_subject(seed):
    s = synth.subject(seed, hash_scale=0.5, res_last_std=0.02)
    s["hash_levels"], s["level_res"], s["log2_T"] = 2, np.array([4, 8], np.uint32), 10
    tab = np.zeros((2, 1 << 10, 2), np.float32)
    rng = np.random.default_rng(seed)
    for l, n in enumerate((4, 8)):
        A = rng.normal(size=(2, 3))
        iz, iy, ix = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
        idx = (ix + iy * (n + 1) + iz * (n + 1) ** 2).ravel()
        tab[l, idx] = (np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1) / n @ A.T).astype(np.float32)
    s["hash_table"] = tab
    return s


def _setup(seed, n_rays=384, S=16):
    subj = _linear_subject(seed)
    frames = synth.training_frames(seed + 1, 3, res=32)
    for c in frames["cameras"]:
        c.n_samples = S
    batch = synth.pixel_batch(seed + 2, n_rays, 3, 32, 32)
    tgt = np.random.default_rng(seed + 3).uniform(0, 1, size=(n_rays, 3)).astype(np.float32)
    return subj, frames, batch, tgt


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_autograd_mse_equals_fused_step():
    nr = nrmod()
    subj, frames, batch, tgt = _setup(101)
    f, px, py, t = u32(batch["frame"]), u32(batch["px"]), u32(batch["py"]), torch.from_numpy(tgt).cuda()
    Sub = nr.Subject(subj)
    try:
        Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
        params = Sub.parameters()
        rgb = nr.RenderFn.apply(Sub, f, px, py, 16, 9, *params)
        loss = ((rgb - t) ** 2).mean()
        loss.backward()
        auto = [p.grad.cpu().numpy().astype(np.float64) for p in params]
        fused_loss = Sub.train_step(f, px, py, t, 16, 9, grad_only=True)
        torch.cuda.synchronize()
        fused = [g.cpu().numpy().astype(np.float64) for g in Sub.parameter_grads()]
    finally:
        Sub.close()
    assert abs(loss.item() - fused_loss) <= 1e-6 * max(1.0, fused_loss)
    for a, b in zip(auto, fused):
        assert np.linalg.norm(b) > 0
        assert _rel(a, b) <= 1e-5


def test_autograd_l1_matches_oracle():
    """A loss only torch knows (mean absolute error): its dL/drgb enters the library's
    compositing adjoint and the parameter gradients match the oracle's autograd."""
    nr = nrmod()
    subj, frames, batch, tgt = _setup(111)
    f, px, py, t = u32(batch["frame"]), u32(batch["px"]), u32(batch["py"]), torch.from_numpy(tgt).cuda()
    Sub = nr.Subject(subj)
    try:
        Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
        params = Sub.parameters()
        rgb = nr.RenderFn.apply(Sub, f, px, py, 16, 13, *params)
        loss = (rgb - t).abs().mean()
        loss.backward()
        got = [p.grad.cpu().numpy().astype(np.float64) for p in params]
    finally:
        Sub.close()
    P = OF.Params(subj, requires_grad=True)
    _, pred = OR.train_loss(subj, P, frames, batch, tgt, 13, 16, np.zeros(3))
    ref_loss = (pred - torch.from_numpy(tgt.astype(np.float64))).abs().mean()
    ref_loss.backward()
    ref = [P.wvol.grad.numpy().ravel(), P.table.grad.numpy().ravel(),
           np.concatenate([np.concatenate([W.grad.numpy().ravel(), b.grad.numpy().ravel()]) for W, b in P.mlp]),
           np.concatenate([np.concatenate([W.grad.numpy().ravel(), b.grad.numpy().ravel()]) for W, b in P.res])]
    assert abs(loss.item() - ref_loss.item()) <= 1e-5
    for g, r, tol in zip(got, ref, (1e-3, 1e-3, 1e-3, 1e-3)):   # the float32 gradient bar
        assert _rel(g, r) <= tol, _rel(g, r)


def test_torch_optimizer_steps_the_library_parameters():
    """torch.optim.Adam over nr parameters (then params_changed) equals the library's own Adam."""
    nr = nrmod()
    subj, frames, batch, tgt = _setup(121)
    f, px, py, t = u32(batch["frame"]), u32(batch["px"]), u32(batch["py"]), torch.from_numpy(tgt).cuda()
    A, B = nr.Subject(subj), nr.Subject(subj)
    try:
        for S in (A, B):
            S.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
        params = A.parameters()
        opt = torch.optim.Adam(params, lr=1e-2, betas=(0.9, 0.99), eps=1e-8)
        rgb = nr.RenderFn.apply(A, f, px, py, 16, 5, *params)
        ((rgb - t) ** 2).mean().backward()
        opt.step()
        A.params_changed()
        B.train_step(f, px, py, t, 16, 5, lr=1e-2)
        torch.cuda.synchronize()
        for pa, pb in zip(A.parameters(), B.parameters()):
            pa, pb = pa.detach().cpu().numpy(), pb.detach().cpu().numpy()
            assert np.abs(pa - pb).max() <= 1e-6 + 1e-5 * np.abs(pb).max()
        cam = frames["cameras"][0]
        A.set_pose(frames["axis_angle"][0], frames["root_t"][0])
        B.set_pose(frames["axis_angle"][0], frames["root_t"][0])
        ia = A.render(cam, nr.make_opts("f32")).cpu().numpy()
        ib = B.render(cam, nr.make_opts("f32")).cpu().numpy()
        assert np.abs(ia - ib).max() <= 1e-5
    finally:
        A.close()
        B.close()
