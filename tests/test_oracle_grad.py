"""Pins of the oracle's gradient (autograd through the FP64 chain) and of its Adam step.

The loss is the squared photometric error of Sec. 2.1 / Sec. 5.2.  Central
finite differences of the oracle's own forward pin the analytic gradient;
torch.optim.Adam pins the update rule (Sec. 5.2: beta = (0.9, 0.99)).
"""
import numpy as np
import pytest
import torch

from oracle import adam
from oracle import field as OF
from oracle import render as OR
from paper_2306_16541_gb300 import synth


def _setup(n_rays=48, n_frames=2):
    subj = synth.subject(21, hash_scale=0.5, res_last_std=0.02)
    frames = synth.training_frames(22, n_frames, res=32)
    for c in frames["cameras"]:
        c.n_samples = 16
    batch = synth.pixel_batch(23, n_rays, n_frames, 32, 32)
    tgt = np.random.default_rng(24).uniform(0, 1, size=(n_rays, 3)).astype(np.float32)
    return subj, frames, batch, tgt


def _fd(subj, P, frames, batch, tgt, ten, j, eps):
    flat = ten.data.reshape(-1)
    old = flat[j].item()
    with torch.no_grad():
        flat[j] = old + eps
        lp, _ = OR.train_loss(subj, P, frames, batch, tgt, 99, 16, np.zeros(3))
        flat[j] = old - eps
        lm, _ = OR.train_loss(subj, P, frames, batch, tgt, 99, 16, np.zeros(3))
        flat[j] = old
    return (lp.item() - lm.item()) / (2 * eps)


def test_gradient_matches_central_differences():
    subj, frames, batch, tgt = _setup()
    P = OF.Params(subj, requires_grad=True)
    loss, _ = OR.train_loss(subj, P, frames, batch, tgt, 99, 16, np.zeros(3))
    loss.backward()
    rng = np.random.default_rng(0)
    groups = {"wvol": P.wvol, "table": P.table, "mlp_W0": P.mlp[0][0], "mlp_Wlast": P.mlp[-1][0],
              "res_W1": P.res[0][0], "res_W4": P.res[3][0], "res_W5": P.res[4][0]}
    eps = 1e-5
    checked = skipped = 0
    for name, ten in groups.items():
        g = ten.grad.reshape(-1)
        nz = torch.nonzero(g.abs() > 1e-9).squeeze(1).numpy()
        if len(nz) == 0:
            continue
        pick = rng.choice(nz, size=min(8, len(nz)), replace=False)
        for j in pick:
            fds = [_fd(subj, P, frames, batch, tgt, ten, j, e) for e in (eps, eps / 10)]
            if abs(fds[0] - fds[1]) > 1e-6 * max(1e-3, abs(fds[0])):
                skipped += 1            # a ReLU, floor or clamp kink lies within eps: not smooth here
                continue
            assert abs(fds[0] - g[j].item()) <= 1e-5 * max(1e-3, abs(fds[0])) + 1e-10, (name, j, fds, g[j].item())
            checked += 1
    assert checked >= 30 and skipped <= checked


def test_adam_matches_torch():
    rng = np.random.default_rng(1)
    p = rng.normal(size=100)
    m = np.zeros(100)
    v = np.zeros(100)
    pt = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-2, betas=(0.9, 0.99), eps=1e-8)
    for k in range(1, 6):
        g = rng.normal(size=100)
        g[::7] = 0.0
        p, m, v = adam.adam_step(p, g, m, v, k, 1e-2)
        pt.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(p, pt.detach().numpy(), atol=1e-14, rtol=0)


@pytest.mark.parametrize("group", ["res", "mlp"])
def test_directional_derivative_along_the_whole_gradient(group):
    """The gradient of a whole MLP (every layer at once) against central differences of the
    loss along its own direction: (L(p + e g/|g|) - L(p - e g/|g|)) / 2e = |g|.  The residual
    MLP moves every sample's canonical point, so the loss is linear in its weights only for
    small steps: at e = 1e-3 in parameter norm the difference quotient already has the wrong
    sign; 1e-5 and 1e-6 are inside the linear range."""
    subj, frames, batch, tgt = _setup()
    P = OF.Params(subj, requires_grad=True)
    loss, _ = OR.train_loss(subj, P, frames, batch, tgt, 99, 16, np.zeros(3))
    loss.backward()
    tens = [t for Wb in (P.res if group == "res" else P.mlp) for t in Wb]
    g = [t.grad.clone() for t in tens]
    nrm = float(torch.sqrt(sum((x ** 2).sum() for x in g)))
    assert nrm > 0
    for eps in (1e-5, 1e-6):
        step = eps / nrm
        with torch.no_grad():
            for t, d in zip(tens, g):
                t.add_(d, alpha=step)
            lp = float(OR.train_loss(subj, P, frames, batch, tgt, 99, 16, np.zeros(3))[0])
            for t, d in zip(tens, g):
                t.add_(d, alpha=-2 * step)
            lm = float(OR.train_loss(subj, P, frames, batch, tgt, 99, 16, np.zeros(3))[0])
            for t, d in zip(tens, g):
                t.add_(d, alpha=step)
        assert abs((lp - lm) / (2 * eps) / nrm - 1.0) <= 1e-2, (group, eps, (lp - lm) / (2 * eps), nrm)
