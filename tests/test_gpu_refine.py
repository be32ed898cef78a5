"""Pose refiner (Sec. 4.1) on the GPU against the FP64 oracle: the refined bone
transforms, rendering with them, the training gradient that flows from every
sample through dL/dG_i and the kinematic chain into MLP_theta, its Adam update,
and serving."""
import numpy as np
import pytest
import torch

from oracle import adam
from oracle import field as OF
from oracle import refine as ORF
from oracle import render as OR
from paper_2306_16541_gb300 import synth

from _util import nrmod

pytestmark = pytest.mark.gpu


def _refiner(seed, width=64, hidden=2, last_std=0.05):
    return synth.refiner_layers(seed, width, hidden, last_std)


def _t64(layers, grad=False):
    return [(torch.from_numpy(W.astype(np.float64)).requires_grad_(grad),
             torch.from_numpy(b.astype(np.float64)).requires_grad_(grad)) for W, b in layers]


def _unpack(flat, layers):
    out, o = [], 0
    for W, b in layers:
        nw, nb = W.size, b.size
        out.append((flat[o:o + nw].reshape(W.shape), flat[o + nw:o + nw + nb]))
        o += nw + nb
    assert o == flat.size
    return out


def _G(R, t):
    return np.concatenate([R, t[:, :, None]], 2).reshape(-1, 12)


@pytest.mark.parametrize("width,hidden", [(64, 2), (256, 4), (40, 1)])
def test_refined_transforms_match_oracle(width, hidden):
    nr = nrmod()
    s = synth.subject(61)
    layers = _refiner(62, width, hidden)
    aa, rt = synth.random_pose(np.random.default_rng(63))
    S = nr.Subject(s)
    try:
        S.set_pose_refiner(layers)
        S.set_pose(aa, rt)
        G = S.pose_transforms()
        S.set_pose_refiner(None)
        G_est = S.pose_transforms()
    finally:
        S.close()
    R, t = ORF.refined_transforms(s["parents"], s["rest_joints"], aa, rt, _t64(layers))
    ref = _G(R.detach().numpy(), t.detach().numpy())
    assert np.abs(G - ref).max() <= 2e-6
    R0, t0 = ORF.refined_transforms(s["parents"], s["rest_joints"], aa, rt, None)
    assert np.abs(G_est - _G(R0.numpy(), t0.numpy())).max() <= 2e-6
    assert np.abs(ref - _G(R0.numpy(), t0.numpy())).max() > 1e-3      # the correction is not trivial


def test_render_with_refiner_matches_oracle():
    nr = nrmod()
    cfg = synth.config_tiny()
    s = synth.subject(64, hash_scale=0.5, res_last_std=0.02)    # MLP_res sees the updated angles
    layers = _refiner(65)
    cam = synth.camera(32, 32, 40.0, (0.0, 0.0, 2.5), 24, 1.5, 3.5)
    S = nr.Subject(s)
    try:
        S.set_pose_refiner(layers)
        S.set_pose(*cfg["pose"])
        img = S.render(cam, nr.make_opts("f32"))
        torch.cuda.synchronize()
        img = img.cpu().numpy().reshape(-1, 4)
    finally:
        S.close()
    py, px = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    ref = OR.render_pixels(s, OF.Params(s), cfg["pose"], cam, px.ravel(), py.ravel(), False,
                           refiner=_t64(layers)).numpy()
    assert np.abs(img - ref).max() <= 1e-3
    assert ref[:, 3].max() > 0.1                       # the performer is in view


def _linear_subject(seed, res_std=0.02):
    """Kink-free encoding (linear dense levels): the gradient has no float32/float64 cell flips.
    A non-zero residual output carries dL/dOmega^o back to the refiner."""
    s = synth.subject(seed, hash_scale=0.5, res_last_std=res_std)
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


def _train(subj, layers, frames, batch, tgt, S_, seed, grad_only, lr=1e-2):
    nr = nrmod()
    Sub = nr.Subject(subj)
    u32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
    try:
        Sub.set_pose_refiner(layers)
        Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
        before = Sub.param(nr.NR_PARAM_REFINER)[0].cpu().numpy().astype(np.float64)
        loss = Sub.train_step(u32(batch["frame"]), u32(batch["px"]), u32(batch["py"]),
                              torch.from_numpy(tgt).cuda(), S_, seed, lr=lr, grad_only=grad_only)
        torch.cuda.synchronize()
        p, g = Sub.param(nr.NR_PARAM_REFINER)
        out = dict(loss=loss, before=before, after=p.cpu().numpy().astype(np.float64),
                   grad=g.cpu().numpy().astype(np.float64),
                   wvol=Sub.param(nr.NR_PARAM_WVOL)[1].cpu().numpy().astype(np.float64))
        return out
    finally:
        Sub.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("n_frames,S_,res_std", [(3, 16, 0.02), (20, 12, 0.02), (3, 16, 0.3)])
def test_refiner_gradient_matches_oracle(n_frames, S_, res_std):
    """dL/dtheta through the per-sample dL/dp_i, the per-frame reduction to dL/dG_i (shared
    memory for up to 16 frames, global atomics beyond), the kinematic chain and MLP_theta,
    plus the residual MLP's conditioning on Omega^o through the rotation log (about 3 % of
    the gradient's norm with the strong residual, 0.4 % with the weak one)."""
    subj = _linear_subject(66, res_std)
    layers = _refiner(67)
    frames = synth.training_frames(68, n_frames, res=32)
    for c in frames["cameras"]:
        c.n_samples = S_
    batch = synth.pixel_batch(69, 512, n_frames, 32, 32)
    tgt = np.random.default_rng(70).uniform(0, 1, size=(512, 3)).astype(np.float32)
    got = _train(subj, layers, frames, batch, tgt, S_, 7, grad_only=True)
    P = OF.Params(subj, requires_grad=True)
    L = _t64(layers, grad=True)
    loss, _ = OR.train_loss(subj, P, frames, batch, tgt, 7, S_, np.zeros(3), refiner=L)
    loss.backward()
    ref = np.concatenate([np.concatenate([W.grad.numpy().ravel(), b.grad.numpy().ravel()]) for W, b in L])
    assert abs(got["loss"] - loss.item()) <= 1e-5 * max(1.0, loss.item())
    assert np.linalg.norm(ref) > 0
    assert _rel(got["grad"], ref) <= 1e-3, _rel(got["grad"], ref)
    assert _rel(got["wvol"], P.wvol.grad.numpy().ravel()) <= 1e-3


def test_refiner_adam_update_and_pose_rederived():
    nr = nrmod()
    subj = _linear_subject(71)
    layers = _refiner(72)
    frames = synth.training_frames(73, 2, res=32)
    for c in frames["cameras"]:
        c.n_samples = 16
    batch = synth.pixel_batch(74, 256, 2, 32, 32)
    tgt = np.random.default_rng(75).uniform(0, 1, size=(256, 3)).astype(np.float32)
    u32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
    aa, rt = synth.random_pose(np.random.default_rng(76))
    Sub = nr.Subject(subj)
    try:
        Sub.set_pose_refiner(layers)
        Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
        Sub.set_pose(aa, rt)
        G0 = Sub.pose_transforms()
        before = Sub.param(nr.NR_PARAM_REFINER)[0].cpu().numpy().astype(np.float64)
        Sub.train_step(u32(batch["frame"]), u32(batch["px"]), u32(batch["py"]), torch.from_numpy(tgt).cuda(),
                       16, 3, lr=1e-2, lr_scale_refiner=0.5)
        torch.cuda.synchronize()
        p, g = Sub.param(nr.NR_PARAM_REFINER)
        after, grad = p.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
        G1 = Sub.pose_transforms()
    finally:
        Sub.close()
    ref, _, _ = adam.adam_step(before, grad, np.zeros_like(grad), np.zeros_like(grad), 1, 5e-3)
    assert np.abs(after - ref).max() <= 1e-6 + 1e-5 * np.abs(ref).max()
    R, t = ORF.refined_transforms(subj["parents"], subj["rest_joints"], aa, rt, _t64(_unpack(after, layers)))
    assert np.abs(G1 - _G(R.detach().numpy(), t.detach().numpy())).max() <= 2e-6
    assert np.abs(G1 - G0).max() > 0


def test_served_request_with_refiner_equals_render():
    nr = nrmod()
    s = synth.subject(77, hash_scale=0.5, res_last_std=0.02, with_ellipsoids=True)
    sub = nr.Subject(s)
    sub.set_pose_refiner(_refiner(78))
    srv = nr.Server(max_bytes=2 << 30, max_slots=2)
    try:
        srv.add_subject(sub)
        rng = np.random.default_rng(79)
        for k in range(3):
            aa, rt = synth.random_pose(rng)
            cam = synth.camera(40, 40, 50.0, synth.random_eye(rng), 24, 0.5, 4.5)
            opts = nr.make_opts(["f32", "bf16", "f32"][k], "f32", k != 2, 1e-4)
            out = torch.full((40, 40, 4), float("nan"), device="cuda")
            srv.wait(srv.submit(srv.request(0, cam, aa, rt, opts, out)), 60000)
            sub.set_pose(aa, rt)
            alone = sub.render(cam, opts)
            torch.cuda.synchronize()
            assert torch.equal(out, alone)
    finally:
        srv.close()
        sub.close()
