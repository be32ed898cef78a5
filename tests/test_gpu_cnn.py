"""CNN_skel (Sec. 4.2) on the GPU against the FP64 oracle: the generated weight
volume (small and full widths), rendering with it, the training gradient from
dL/dW^c through the softmax and the five transposed convolutions, and the Adam
step followed by regeneration."""
import numpy as np
import pytest
import torch

from oracle import adam
from oracle import cnn
from oracle import field as OF
from oracle import render as OR
from paper_2306_16541_gb300 import synth

from _util import nrmod

pytestmark = pytest.mark.gpu

SMALL = (16, 16, 8, 8, 8)


def _prior(subj):
    return np.log(np.asarray(subj["wvol"], np.float64) + 1e-6).astype(np.float32)


def _oracle_volume(layers, z, prior):
    return cnn.weight_volume(cnn.as_tensors(layers), torch.from_numpy(z.astype(np.float64)),
                             None if prior is None else torch.from_numpy(prior.astype(np.float64))).numpy()


def _gpu_volume(S, nr):
    # any consumer regenerates the volume: a one-point query is the cheapest
    S.query(torch.zeros(1, 3, device="cuda"))
    torch.cuda.synchronize()
    return S.param(nr.NR_PARAM_WVOL)[0].cpu().numpy().reshape(25, 32, 32, 32)


@pytest.mark.parametrize("channels,with_prior", [(SMALL, True), (SMALL, False), ((1024, 512, 256, 128, 64), True)])
def test_generated_volume_matches_oracle(channels, with_prior):
    nr = nrmod()
    s = synth.subject(81)
    layers = synth.cnn_layers(82, channels, last_std=0.3)
    z = synth.cnn_latent(83)
    prior = _prior(s) if with_prior else None
    S = nr.Subject(s)
    try:
        S.set_pose(*synth.random_pose(np.random.default_rng(84)))
        S.set_weight_cnn(layers, z, prior)
        got = _gpu_volume(S, nr)
    finally:
        S.close()
    ref = _oracle_volume(layers, z, prior)
    assert np.abs(got - ref).max() <= 1e-5 + 1e-4 * np.abs(ref).max()
    assert np.allclose(got.sum(0), 1.0, atol=1e-5)


def test_render_with_generated_volume_matches_oracle():
    nr = nrmod()
    s = synth.subject(85, hash_scale=0.5, res_last_std=0.02)
    layers = synth.cnn_layers(86, SMALL, last_std=0.1)
    z = synth.cnn_latent(87)
    prior = _prior(s)
    pose = synth.random_pose(np.random.default_rng(88))
    cam = synth.camera(32, 32, 40.0, (0.0, 0.0, 2.5), 24, 1.5, 3.5)
    S = nr.Subject(s)
    try:
        S.set_weight_cnn(layers, z, prior)
        S.set_pose(*pose)
        img = S.render(cam, nr.make_opts("f32"))
        torch.cuda.synchronize()
        img = img.cpu().numpy().reshape(-1, 4)
    finally:
        S.close()
    s2 = dict(s)
    s2["wvol"] = _oracle_volume(layers, z, prior)
    py, px = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    ref = OR.render_pixels(s2, OF.Params(s2), pose, cam, px.ravel(), py.ravel(), False).numpy()
    assert np.abs(img - ref).max() <= 1e-3
    assert ref[:, 3].max() > 0.1


def _linear_subject(seed):
    s = synth.subject(seed, hash_scale=0.5)
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("lr", [0.0, 1e-3])
def test_generator_gradient_and_adam_step_match_oracle(lr):
    """lr 0: gradient only; lr > 0: one Adam step on the generator, after which the
    volume is regenerated from the updated weights."""
    nr = nrmod()
    subj = _linear_subject(89)
    layers = synth.cnn_layers(90, SMALL, last_std=0.3)
    z = synth.cnn_latent(91)
    prior = _prior(synth.subject(89))
    frames = synth.training_frames(92, 3, res=32)
    for c in frames["cameras"]:
        c.n_samples = 16
    batch = synth.pixel_batch(93, 512, 3, 32, 32)
    tgt = np.random.default_rng(94).uniform(0, 1, size=(512, 3)).astype(np.float32)
    u32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
    Sub = nr.Subject(subj)
    try:
        Sub.set_weight_cnn(layers, z, prior)
        Sub.set_pose(*synth.random_pose(np.random.default_rng(95)))
        Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
        before = Sub.param(nr.NR_PARAM_CNN)[0].cpu().numpy().astype(np.float64)
        loss = Sub.train_step(u32(batch["frame"]), u32(batch["px"]), u32(batch["py"]), torch.from_numpy(tgt).cuda(),
                              16, 5, lr=lr if lr > 0 else 1e-2, grad_only=lr == 0.0,
                              train_mask=nr.NR_TRAIN_CNN if lr > 0 else 0)
        torch.cuda.synchronize()
        p, g = Sub.param(nr.NR_PARAM_CNN)
        after, grad = p.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
        vol_after = _gpu_volume(Sub, nr) if lr > 0 else None
    finally:
        Sub.close()
    L = cnn.as_tensors(layers, requires_grad=True)
    P = OF.Params(subj)
    P.wvol = cnn.weight_volume(L, torch.from_numpy(z.astype(np.float64)), torch.from_numpy(prior.astype(np.float64)))
    ref_loss, _ = OR.train_loss(subj, P, frames, batch, tgt, 5, 16, np.zeros(3))
    ref_loss.backward()
    ref = np.concatenate([np.concatenate([W.grad.numpy().ravel(), b.grad.numpy().ravel()]) for W, b in L])
    assert abs(loss - ref_loss.item()) <= 1e-5 * max(1.0, ref_loss.item())
    assert np.linalg.norm(ref) > 0
    assert _rel(grad, ref) <= 1e-3, _rel(grad, ref)
    if lr > 0:
        upd, _, _ = adam.adam_step(before, grad, np.zeros_like(grad), np.zeros_like(grad), 1, lr)
        assert np.abs(after - upd).max() <= 1e-6 + 1e-5 * np.abs(upd).max()
        flat, o, new = after.astype(np.float32), 0, []
        for W, b in layers:
            new.append((flat[o:o + W.size].reshape(W.shape), flat[o + W.size:o + W.size + b.size]))
            o += W.size + b.size
        ref_vol = _oracle_volume(new, z, prior)
        assert np.abs(vol_after - ref_vol).max() <= 1e-5 + 1e-4 * np.abs(ref_vol).max()
