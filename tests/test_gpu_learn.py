"""What training buys: the trained field against the untrained one on held-out
frames, and the trained non-rigid residual (Sec. 4.3) against the same training
with the residual frozen, on a performer whose motion has a non-rigid part.

Targets are rendered from a seeded ground-truth subject (textured hash entries
U(-0.5, 0.5), a density bias of 3, a non-zero residual MLP); the trainee shares its skeleton and
starts from the initial state of the tiny workload (hash entries U(-1e-4, 1e-4),
other MLP weights, the residual's output layer at zero).  Adam at lr 1e-2 for the
canonical field and 1e-3 for the weight volume and the residual MLP (Sec. 5.2 trains
the networks other than the NeRF network at a 10x smaller rate).
"""
import numpy as np
import pytest
import torch

from paper_2306_16541_gb300 import synth

from _util import nrmod, psnr

pytestmark = pytest.mark.gpu

RES, S, N_TRAIN, N_TEST = 48, 48, 12, 4


def _frames(seed, n):
    fr = synth.training_frames(seed, n, res=RES)
    for c in fr["cameras"]:
        c.n_samples = S
    return fr


def _render_set(nr, subj, frames):
    Sub = nr.Subject(subj)
    try:
        imgs = []
        for i, cam in enumerate(frames["cameras"]):
            Sub.set_pose(frames["axis_angle"][i], frames["root_t"][i])
            imgs.append(Sub.render(cam, nr.make_opts("f32")).clone())
        return torch.stack(imgs)
    finally:
        Sub.close()


def _train(nr, subj, frames, targets, steps, mask=0, seed=0):
    Sub = nr.Subject(subj)
    Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
    g = torch.Generator(device="cuda").manual_seed(seed)
    n = 4096
    losses = []
    for k in range(steps):
        f = torch.randint(0, len(frames["cameras"]), (n,), device="cuda", generator=g, dtype=torch.int32)
        px = torch.randint(0, RES, (n,), device="cuda", generator=g, dtype=torch.int32)
        py = torch.randint(0, RES, (n,), device="cuda", generator=g, dtype=torch.int32)
        tgt = targets[f.long(), py.long(), px.long(), :3].contiguous()
        losses.append(Sub.train_step(f, px, py, tgt, S, 1000 + k, lr=1e-2, train_mask=mask,
                                     lr_scale=nr.PAPER_LR_SCALE))
    return Sub, losses


def _eval(nr, Sub, frames, targets):
    out = []
    for i, cam in enumerate(frames["cameras"]):
        Sub.set_pose(frames["axis_angle"][i], frames["root_t"][i])
        out.append(psnr(Sub.render(cam, nr.make_opts("f32")).cpu().numpy()[..., :3],
                        targets[i, ..., :3].cpu().numpy()))
    return float(np.mean(out))


def _subjects():
    gt = synth.subject(500, hash_scale=0.5, res_last_std=0.03)
    gt["mlp_layers"][-1][1][3] = 3.0            # a visible, mostly opaque performer
    gt["mlp_params"] = synth.pack_layers(gt["mlp_layers"])
    trainee = synth.subject(500)
    other = synth.subject(501)
    trainee["mlp_layers"], trainee["mlp_params"] = other["mlp_layers"], other["mlp_params"]
    return gt, trainee


def test_training_improves_held_out_frames():
    nr = nrmod()
    gt, trainee = _subjects()
    train_fr, test_fr = _frames(600, N_TRAIN), _frames(601, N_TEST)
    train_tg, test_tg = _render_set(nr, gt, train_fr), _render_set(nr, gt, test_fr)
    Sub0 = nr.Subject(trainee)
    before = _eval(nr, Sub0, test_fr, test_tg)
    Sub0.close()
    Sub, losses = _train(nr, trainee, train_fr, train_tg, 300)
    after = _eval(nr, Sub, test_fr, test_tg)
    Sub.close()
    print(f"held-out PSNR: untrained {before:.2f} dB, trained {after:.2f} dB; loss {losses[0]:.4g} -> {losses[-1]:.4g}")
    assert losses[-1] < 0.25 * losses[0]
    assert after >= before + 6.0


def test_residual_training_on_non_rigid_motion_is_measured():
    """MLP_res (Sec. 4.3) trained against the same training with it frozen, on a performer whose
    motion has a non-rigid part.  No held-out gain appears on these synthetic performers (the
    measured figures and the reason -- the loss is linear in MLP_res's weights only within
    ~1e-4 of parameter norm, below one Adam step -- are reported with the design); what is
    asserted is the mechanism: the frozen run leaves MLP_res bit for bit as it was, the trained
    run moves it, and both fits are sound."""
    nr = nrmod()
    gt, trainee = _subjects()
    train_fr, test_fr = _frames(610, N_TRAIN), _frames(611, N_TEST)
    train_tg, test_tg = _render_set(nr, gt, train_fr), _render_set(nr, gt, test_fr)
    res0 = np.asarray(trainee["res_params"], np.float32)
    out = {}
    for name, mask in (("trained", nr.NR_TRAIN_ALL), ("frozen", nr.NR_TRAIN_ALL & ~nr.NR_TRAIN_RES)):
        Sub, losses = _train(nr, trainee, train_fr, train_tg, 300, mask=mask, seed=1)
        res = Sub.param(nr.NR_PARAM_RES)[0].cpu().numpy()
        out[name] = (_eval(nr, Sub, train_fr, train_tg), _eval(nr, Sub, test_fr, test_tg), res, losses)
        Sub.close()
    print("residual trained: training frames %.2f dB, held-out %.2f dB; frozen: %.2f dB, %.2f dB"
          % (out["trained"][0], out["trained"][1], out["frozen"][0], out["frozen"][1]))
    assert np.array_equal(out["frozen"][2], res0)
    assert np.abs(out["trained"][2] - res0).max() > 0
    for name in out:
        assert np.isfinite(out[name][3]).all() and out[name][3][-1] < 0.25 * out[name][3][0]
        assert out[name][1] > 25.0


def _train_refined(nr, subj, frames, targets, steps, refiner, seed=0):
    Sub = nr.Subject(subj)
    if refiner is not None:
        Sub.set_pose_refiner(refiner)
    Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
    g = torch.Generator(device="cuda").manual_seed(seed)
    n = 4096
    for k in range(steps):
        f = torch.randint(0, len(frames["cameras"]), (n,), device="cuda", generator=g, dtype=torch.int32)
        px = torch.randint(0, RES, (n,), device="cuda", generator=g, dtype=torch.int32)
        py = torch.randint(0, RES, (n,), device="cuda", generator=g, dtype=torch.int32)
        tgt = targets[f.long(), py.long(), px.long(), :3].contiguous()
        Sub.train_step(f, px, py, tgt, S, 2000 + k, lr=1e-2, lr_scale=nr.PAPER_LR_SCALE, lr_scale_refiner=0.1)
    return Sub


def test_pose_refiner_corrects_noisy_pose_estimates():
    """Sec. 4.1: the training frames come with pose estimates off by ~6 degrees per joint (the
    targets were rendered with the true poses).  Trained with MLP_theta, the canonical field
    stays consistent across frames; trained without it, the field blurs to fit the wrong poses.
    Measured on held-out frames rendered at their true poses (refiner off for both)."""
    nr = nrmod()
    gt, trainee = _subjects()
    true_fr, test_fr = _frames(620, N_TRAIN), _frames(623, N_TEST)
    targets, test_tg = _render_set(nr, gt, true_fr), _render_set(nr, gt, test_fr)
    noisy = dict(true_fr)
    rng = np.random.default_rng(621)
    aa = np.array(true_fr["axis_angle"], np.float32, copy=True)
    aa[:, 1:] += rng.normal(scale=0.1, size=aa[:, 1:].shape).astype(np.float32)
    noisy["axis_angle"] = aa
    results = {}
    for name, ref in (("refined", synth.refiner_layers(622, 128, 2)), ("plain", None)):
        Sub = _train_refined(nr, trainee, noisy, targets, 400, ref, seed=3)
        train_psnr = _eval(nr, Sub, noisy, targets)
        Sub.set_pose_refiner(None)
        results[name] = _eval(nr, Sub, test_fr, test_tg)
        print(f"{name}: training frames {train_psnr:.2f} dB, held-out true poses {results[name]:.2f} dB")
        Sub.close()
    assert results["refined"] >= results["plain"] + 3.0        # measured: 32.4 vs 24.2 dB
