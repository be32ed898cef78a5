"""Training step parity (Sec. 5.2): loss, hand-written gradients and the Adam update
of the CUDA path against the FP64 oracle (autograd through the oracle's chain,
itself pinned by central differences in test_oracle_grad.py)."""
import numpy as np
import pytest
import torch

from oracle import adam
from oracle import field as OF
from oracle import render as OR
from paper_2306_16541_gb300 import synth

from _util import nrmod

pytestmark = pytest.mark.gpu

GROUPS = ["wvol", "table", "mlp", "res"]


def u32(a):
    """uint32 indices as an int32 CUDA tensor with the same bits."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _smooth(subj):
    """Level-l table entries scaled by (16 / N_l)^2: coarse levels dominate.

    The hash interpolation is only C0 and the MLPs are piecewise linear, so a
    sample's gradient jumps where it crosses a cell face or a ReLU kink.  The
    float32 and float64 sides place a sample ~1e-7 apart; where that straddles a
    kink the two gradients differ by O(1) for that sample, and a sample whose
    bone-weight sum S is below the 1e-4 floor multiplies dL/dx_skel by 1 / 1e-4
    in its weight-volume gradient.  A coarse-dominated field keeps such flips out
    of the comparison; the formula is the same everywhere.
    """
    s = dict(subj)
    lv = np.asarray(s["level_res"], np.float32)
    s["hash_table"] = (s["hash_table"] * (16.0 / lv[:, None, None]) ** 2).astype(np.float32)
    return s


def _setup(n_rays=384, n_frames=3, res=32, S=16, seed=31):
    subj = _smooth(synth.subject(seed, hash_scale=0.5, res_last_std=0.02))
    frames = synth.training_frames(seed + 1, n_frames, res=res)
    for c in frames["cameras"]:
        c.n_samples = S
    batch = synth.pixel_batch(seed + 2, n_rays, n_frames, res, res)
    tgt = np.random.default_rng(seed + 3).uniform(0, 1, size=(n_rays, 3)).astype(np.float32)
    return subj, frames, batch, tgt


def _gpu_step(subj, frames, batch, tgt, S, seed, grad_only, lr=1e-2, train_mask=0, loss_weight=0.0):
    nr = nrmod()
    Sub = nr.Subject(subj)
    try:
        Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
        before = {g: Sub.param(i)[0].clone() for i, g in enumerate(GROUPS)}
        loss = Sub.train_step(u32(batch["frame"]), u32(batch["px"]), u32(batch["py"]),
                              torch.from_numpy(np.ascontiguousarray(tgt, np.float32)).cuda(), S, seed,
                              lr=lr, grad_only=grad_only, train_mask=train_mask, loss_weight=loss_weight)
        torch.cuda.synchronize()
        grads = {g: Sub.param(i)[1].cpu().numpy().astype(np.float64) for i, g in enumerate(GROUPS)}
        after = {g: Sub.param(i)[0].cpu().numpy().astype(np.float64) for i, g in enumerate(GROUPS)}
        before = {g: v.cpu().numpy().astype(np.float64) for g, v in before.items()}
        return loss, grads, before, after
    finally:
        Sub.close()


def _oracle_grads(subj, frames, batch, tgt, S, seed, loss_weight=1.0):
    P = OF.Params(subj, requires_grad=True)
    loss, _ = OR.train_loss(subj, P, frames, batch, tgt, seed, S, np.zeros(3), loss_weight=loss_weight)
    loss.backward()
    g = {"wvol": P.wvol.grad.numpy().ravel(), "table": P.table.grad.numpy().ravel()}
    g["mlp"] = np.concatenate([np.concatenate([W.grad.numpy().ravel(), b.grad.numpy().ravel()]) for W, b in P.mlp])
    g["res"] = np.concatenate([np.concatenate([W.grad.numpy().ravel(), b.grad.numpy().ravel()]) for W, b in P.res])
    return float(loss.item()), g


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


# Relative L2 bounds per group.  The weight volume's bound is looser: a sample
# whose bone-weight sum S lies under the 1e-4 floor moves its canonical point
# by p_i / 1e-4 per unit weight, so a float32-vs-float64 ReLU or cell-face flip
# at such a sample shifts many voxel gradients at once (see _smooth).  Measured
# on this batch: 4.5e-3 (the other groups 4e-7 .. 6e-5).
TOL = {"wvol": 6e-3, "table": 1e-3, "mlp": 1e-3, "res": 1e-3}


def test_gradients_match_oracle():
    subj, frames, batch, tgt = _setup()
    loss, grads, _, _ = _gpu_step(subj, frames, batch, tgt, 16, 77, grad_only=True)
    ref_loss, ref = _oracle_grads(subj, frames, batch, tgt, 16, 77)
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, ref_loss), (loss, ref_loss)
    print("relative L2 per group:", {g: _rel(grads[g], ref[g]) for g in GROUPS})
    for g in GROUPS:
        assert np.linalg.norm(ref[g]) > 0, g
        assert _rel(grads[g], ref[g]) <= TOL[g], (g, _rel(grads[g], ref[g]))


def test_rays_longer_than_a_block_take_the_separate_kernels():
    """A step whose rays hold more samples than a backward block has threads (400 > 384) runs the
    forward, the compositing adjoint and the backward as separate kernels (the backward
    recomputing the forward); its loss and gradients meet the same bounds against the oracle."""
    subj, frames, batch, tgt = _setup(n_rays=48, S=400, seed=33)
    loss, grads, _, _ = _gpu_step(subj, frames, batch, tgt, 400, 79, grad_only=True)
    ref_loss, ref = _oracle_grads(subj, frames, batch, tgt, 400, 79)
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, ref_loss), (loss, ref_loss)
    print("S = 400: relative L2 per group:", {g: _rel(grads[g], ref[g]) for g in GROUPS})
    for g in GROUPS:
        assert np.linalg.norm(ref[g]) > 0, g
        assert _rel(grads[g], ref[g]) <= TOL[g], (g, _rel(grads[g], ref[g]))


def _linear_table(subj, levels=(4, 8), log2_t=10, seed=0):
    """Dense levels holding a linear function of the vertex position: the encoding is
    linear in x_final, with no kink at cell faces."""
    s = dict(subj)
    s["hash_levels"], s["level_res"], s["log2_T"] = len(levels), np.array(levels, np.uint32), log2_t
    tab = np.zeros((len(levels), 1 << log2_t, 2), np.float32)
    rng = np.random.default_rng(seed)
    for l, n in enumerate(levels):
        A = rng.normal(size=(2, 3))
        iz, iy, ix = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
        idx = (ix + iy * (n + 1) + iz * (n + 1) ** 2).ravel()
        tab[l, idx] = (np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1) / n @ A.T).astype(np.float32)
    s["hash_table"] = tab
    return s


def test_weight_volume_gradient_on_a_kink_free_field():
    """Linear encoding and a zero residual output: dL/dx_skel has no float32/float64
    kink flips, so the inverse-LBS scatter-add is compared tightly."""
    subj = _linear_table(synth.subject(31, hash_scale=0.5))
    frames = synth.training_frames(32, 3, res=32)
    for c in frames["cameras"]:
        c.n_samples = 16
    batch = synth.pixel_batch(33, 384, 3, 32, 32)
    tgt = np.random.default_rng(34).uniform(0, 1, size=(384, 3)).astype(np.float32)
    loss, grads, _, _ = _gpu_step(subj, frames, batch, tgt, 16, 77, grad_only=True)
    ref_loss, ref = _oracle_grads(subj, frames, batch, tgt, 16, 77)
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, ref_loss)
    for g in ("wvol", "table", "mlp"):
        assert _rel(grads[g], ref[g]) <= 1e-4, (g, _rel(grads[g], ref[g]))


def test_aggregated_scatter_adds_over_whole_warp_runs():
    """128 samples per ray put each warp on 32 consecutive samples of one ray, and the
    0.5 m cells of a resolution-4 level hold runs of up to 32 lanes: the warp-aggregated
    scatter-adds (run sums over shuffles, one atomic per run) against the oracle, tightly,
    on the kink-free field."""
    subj = _linear_table(synth.subject(35, hash_scale=0.5))
    frames = synth.training_frames(36, 2, res=32)
    for c in frames["cameras"]:
        c.n_samples = 128
    batch = synth.pixel_batch(37, 48, 2, 32, 32)
    tgt = np.random.default_rng(38).uniform(0, 1, size=(48, 3)).astype(np.float32)
    loss, grads, _, _ = _gpu_step(subj, frames, batch, tgt, 128, 79, grad_only=True)
    ref_loss, ref = _oracle_grads(subj, frames, batch, tgt, 128, 79)
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, ref_loss)
    for g in ("wvol", "table", "mlp"):
        assert np.linalg.norm(ref[g]) > 0, g
        assert _rel(grads[g], ref[g]) <= 1e-4, (g, _rel(grads[g], ref[g]))


def test_gradients_with_hann_window_and_more_samples():
    subj, frames, batch, tgt = _setup(n_rays=200, n_frames=2, S=40, seed=41)
    nr = nrmod()
    # partial window: bands beyond alpha are damped (Sec. 4.3 coarse-to-fine schedule)
    Sub = nr.Subject(subj)
    try:
        Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
        loss = Sub.train_step(u32(batch["frame"]), u32(batch["px"]), u32(batch["py"]),
                              torch.from_numpy(tgt).cuda(), 40, 5, grad_only=True, hann_alpha=2.5)
        torch.cuda.synchronize()
        gres = Sub.param(3)[1].cpu().numpy().astype(np.float64)
    finally:
        Sub.close()
    P = OF.Params(subj, requires_grad=True)
    ref_loss, _ = OR.train_loss(subj, P, frames, batch, tgt, 5, 40, np.zeros(3), alpha=2.5)
    ref_loss.backward()
    ref = np.concatenate([np.concatenate([W.grad.numpy().ravel(), b.grad.numpy().ravel()]) for W, b in P.res])
    assert abs(loss - ref_loss.item()) <= 1e-5 * max(1.0, ref_loss.item())
    assert _rel(gres, ref) <= 1e-3


def test_adam_update_matches_oracle_rule():
    subj, frames, batch, tgt = _setup(n_rays=256, seed=51)
    loss, grads, before, after = _gpu_step(subj, frames, batch, tgt, 16, 9, grad_only=False, lr=1e-2)
    for g in GROUPS:
        ref, _, _ = adam.adam_step(before[g], grads[g], np.zeros_like(grads[g]), np.zeros_like(grads[g]), 1, 1e-2)
        assert np.abs(after[g] - ref).max() <= 1e-6 + 1e-5 * np.abs(ref).max(), g


def test_train_mask_freezes_groups():
    subj, frames, batch, tgt = _setup(n_rays=128, seed=61)
    nr = nrmod()
    _, _, before, after = _gpu_step(subj, frames, batch, tgt, 16, 3, grad_only=False,
                                    train_mask=nr.NR_TRAIN_HASH | nr.NR_TRAIN_MLP)
    assert np.array_equal(before["wvol"], after["wvol"]) and np.array_equal(before["res"], after["res"])
    assert not np.array_equal(before["table"], after["table"]) and not np.array_equal(before["mlp"], after["mlp"])


def test_patch_batch_with_weighted_mse():
    """Sec. 5.2 batch layout: 6 patches of 20 x 20 pixels per image, the MSE term
    weighted by lambda_mse = 0.2; loss and gradients against the oracle on the
    kink-free linear-table field (2400 contiguous rays put many samples near
    the same cell faces, where float32 and float64 may pick different cells)."""
    nr = nrmod()
    subj = _linear_table(synth.subject(71, hash_scale=0.5))
    frames = synth.training_frames(72, 4, res=48)
    for c in frames["cameras"]:
        c.n_samples = 16
    batch = synth.patch_batch(73, 4, n_images=1, width=48, height=48)
    n = batch["frame"].shape[0]
    assert n == 6 * 400
    tgt = np.random.default_rng(74).uniform(0, 1, size=(n, 3)).astype(np.float32)
    loss, grads, _, _ = _gpu_step(subj, frames, batch, tgt, 16, 19, grad_only=True,
                                  loss_weight=nr.PAPER_MSE_WEIGHT)
    ref_loss, ref = _oracle_grads(subj, frames, batch, tgt, 16, 19, loss_weight=nr.PAPER_MSE_WEIGHT)
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, ref_loss), (loss, ref_loss)
    for g in ("wvol", "table", "mlp"):
        assert np.linalg.norm(ref[g]) > 0, g
        assert _rel(grads[g], ref[g]) <= 1e-4, (g, _rel(grads[g], ref[g]))


def _per_tensor(flat, layers):
    """Splits a flat master array [W1, b1, W2, b2, ...] into the tensors of `layers`."""
    out, o = [], 0
    for W, b in layers:
        nW, nb = int(np.prod(np.shape(W))), int(np.prod(np.shape(b)))
        out.append((flat[o:o + nW], flat[o + nW:o + nW + nb]))
        o += nW + nb
    assert o == flat.size
    return out


@pytest.mark.parametrize("last_std", [0.02, 0.0])
def test_every_mlp_tensor_gradient_matches_oracle(last_std):
    """Per weight matrix and bias vector, not per group: a group's norm is dominated by its
    largest tensor (the residual MLP's output layer), so an error confined to an inner layer or
    to the pose columns of residual layer 1 would hide under a group-level bound.  A non-zero
    residual output layer gives every residual layer a gradient; a zero one (the initial state)
    leaves gradient only on the output layer, which must then match alone.  (With a residual
    whose offsets reach decimetres, float32-vs-float64 kink flips at the moved canonical points
    put every residual tensor ~2 % off; the workloads' residuals stay at centimetres.)"""
    subj = _smooth(synth.subject(35, hash_scale=0.5, res_last_std=last_std if last_std > 0 else None))
    frames = synth.training_frames(36, 3, res=32)
    for c in frames["cameras"]:
        c.n_samples = 16
    batch = synth.pixel_batch(37, 384, 3, 32, 32)
    tgt = np.random.default_rng(38).uniform(0, 1, size=(384, 3)).astype(np.float32)
    _, grads, _, _ = _gpu_step(subj, frames, batch, tgt, 16, 77, grad_only=True)
    P = OF.Params(subj, requires_grad=True)
    loss, _ = OR.train_loss(subj, P, frames, batch, tgt, 77, 16, np.zeros(3))
    loss.backward()
    g_dims = 3 + 6 * int(subj["res_pe_freqs"])
    for name, layers, flat in (("res", P.res, grads["res"]), ("mlp", P.mlp, grads["mlp"])):
        got = _per_tensor(flat, [(W.detach().numpy(), b.detach().numpy()) for W, b in layers])
        for k, ((W, b), (gW, gb)) in enumerate(zip(layers, got)):
            for what, ref, val in (("W", W.grad.numpy().ravel(), gW), ("b", b.grad.numpy().ravel(), gb)):
                if np.linalg.norm(ref) == 0:
                    assert np.abs(val).max() <= 1e-12, (name, k, what)
                    continue
                assert _rel(val, ref) <= 2e-3, (name, k + 1, what, _rel(val, ref))
            if name == "res" and k == 0 and np.linalg.norm(W.grad.numpy()[:, g_dims:]) > 0:
                # the pose columns (Omega joins layer 1 as a per-frame bias on the device)
                ref = W.grad.numpy()[:, g_dims:].ravel()
                val = gW.reshape(W.shape)[:, g_dims:].ravel()
                assert _rel(val, ref) <= 2e-3, ("res pose columns", _rel(val, ref))
