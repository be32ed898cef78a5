"""Pins of the oracle's CNN_skel weight-volume generator (Sec. 4.2): the
transposed convolution against a brute-force scatter, the generator's shape
and partition of unity, and central differences of the loss in its weights."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import cnn
from oracle import field as OF
from oracle import render as OR
from paper_2306_16541_gb300 import synth


def test_transposed_convolution_matches_brute_force_scatter():
    """Kernel 4, stride 2, padding 1: input voxel i adds x[i] W[k] to output 2 i - 1 + k."""
    rng = np.random.default_rng(0)
    Ci, Co, r = 3, 2, 3
    x = rng.normal(size=(Ci, r, r, r))
    W = rng.normal(size=(Ci, Co, 4, 4, 4))
    b = rng.normal(size=Co)
    R = 2 * r
    ref = np.zeros((Co, R, R, R)) + b[:, None, None, None]
    for i in range(Ci):
        for z in range(r):
            for y in range(r):
                for xx in range(r):
                    for kz in range(4):
                        for ky in range(4):
                            for kx in range(4):
                                uz, uy, ux = 2 * z - 1 + kz, 2 * y - 1 + ky, 2 * xx - 1 + kx
                                if 0 <= uz < R and 0 <= uy < R and 0 <= ux < R:
                                    ref[:, uz, uy, ux] += x[i, z, y, xx] * W[i, :, kz, ky, kx]
    got = F.conv_transpose3d(torch.from_numpy(x)[None], torch.from_numpy(W), torch.from_numpy(b), stride=2, padding=1)
    assert np.allclose(got[0].numpy(), ref, atol=1e-12)


def test_generator_shape_and_partition_of_unity():
    layers = cnn.as_tensors(synth.cnn_layers(1, (16, 8, 8, 4, 4), last_std=0.5))
    z = torch.from_numpy(synth.cnn_latent(2).astype(np.float64))
    W = cnn.weight_volume(layers, z)
    assert W.shape == (25, 32, 32, 32)
    assert torch.allclose(W.sum(0), torch.ones(32, 32, 32, dtype=torch.float64), atol=1e-14)
    assert float(W.min()) > 0 and float(W.std()) > 1e-3
    prior = np.random.default_rng(3).dirichlet(np.ones(25), size=32 ** 3).T.reshape(25, 32, 32, 32)
    zero = [(torch.zeros_like(Wt), torch.zeros_like(bt)) for Wt, bt in layers]
    Wp = cnn.weight_volume(zero, z, torch.from_numpy(np.log(prior)))
    assert np.allclose(Wp.numpy(), prior, atol=1e-12)       # zero network: the prior itself


def test_loss_gradient_in_generator_weights_matches_central_differences():
    subj = synth.subject(31, hash_scale=0.5)
    frames = synth.training_frames(32, 2, res=24)
    for c in frames["cameras"]:
        c.n_samples = 12
    batch = synth.pixel_batch(33, 40, 2, 24, 24)
    tgt = np.random.default_rng(34).uniform(0, 1, size=(40, 3)).astype(np.float32)
    layers = cnn.as_tensors(synth.cnn_layers(35, (8, 8, 4, 4, 4), last_std=0.3), requires_grad=True)
    z = torch.from_numpy(synth.cnn_latent(36).astype(np.float64))
    prior = torch.from_numpy(np.log(np.asarray(subj["wvol"], np.float64) + 1e-6))

    def loss_fn():
        P = OF.Params(subj)
        P.wvol = cnn.weight_volume(layers, z, prior)
        return OR.train_loss(subj, P, frames, batch, tgt, 5, 12, np.zeros(3))[0]

    loss = loss_fn()
    loss.backward()
    rng = np.random.default_rng(0)
    checked = skipped = 0
    for ten in (layers[0][0], layers[2][0], layers[5][0], layers[5][1]):
        g = ten.grad.reshape(-1)
        nz = torch.nonzero(g.abs() > 1e-10).squeeze(1).numpy()
        for j in rng.choice(nz, size=min(6, len(nz)), replace=False):
            flat = ten.data.reshape(-1)
            old = flat[j].item()
            fds = []
            for e in (1e-5, 1e-6):
                with torch.no_grad():
                    flat[j] = old + e
                    lp = loss_fn().item()
                    flat[j] = old - e
                    lm = loss_fn().item()
                    flat[j] = old
                fds.append((lp - lm) / (2 * e))
            if abs(fds[0] - fds[1]) > 1e-6 * max(1e-3, abs(fds[0])):
                skipped += 1
                continue
            assert abs(fds[0] - g[j].item()) <= 1e-5 * max(1e-3, abs(fds[0])) + 1e-11
            checked += 1
    assert checked >= 12 and skipped <= checked, (checked, skipped)
