"""Pins of the oracle's pose refiner (Sec. 4.1) and its differentiable forward
kinematics: the numpy Rodrigues map and FK (themselves pinned against direct
products), the closed-form derivative of the rotation at zero, scipy's rotation
composition, and central differences of the loss in the refiner's weights."""
import numpy as np
import pytest
import torch

from oracle import fk
from oracle import field as OF
from oracle import refine
from oracle import render as OR
from paper_2306_16541_gb300 import synth


def _layers(seed, last_std=0.05, width=32, hidden=2):
    return [(torch.from_numpy(W.astype(np.float64)), torch.from_numpy(b.astype(np.float64)))
            for W, b in synth.refiner_layers(seed, width, hidden, last_std)]


def test_rodrigues_matches_numpy_form():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(size=(20, 3)), 1e-9 * rng.normal(size=(5, 3)), np.zeros((1, 3))])
    assert np.allclose(refine.rodrigues_t(torch.from_numpy(v)).numpy(), fk.rodrigues(v), atol=1e-14, rtol=0)


def test_rotation_derivative_at_zero_is_the_generator():
    """d Rot(v) / d v_a at v = 0 is [e_a]_x (the so(3) generator)."""
    v = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    J = torch.autograd.functional.jacobian(refine.rodrigues_t, v)      # [3, 3, 3]
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1.0
        gen = np.array([[0, -e[2], e[1]], [e[2], 0, -e[0]], [-e[1], e[0], 0]])
        assert np.allclose(J[:, :, a].numpy(), gen, atol=1e-15)


def test_rotation_log_matches_scipy_and_inverts_rodrigues():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(9)
    axis = rng.normal(size=(30, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = np.concatenate([rng.uniform(0, 3.0, 25), [1e-9, 1e-6, 1e-4, 0.0, 2.9]])
    v = axis * ang[:, None]
    R = fk.rodrigues(v)
    got = refine.rot_log_t(torch.from_numpy(R)).numpy()
    assert np.allclose(got, Rot.from_matrix(R).as_rotvec(), atol=1e-9)
    assert np.allclose(got, v, atol=1e-9)


def test_updated_angles_of_a_fixed_correction():
    """Omega^o of joint j >= 1 is the rotation vector of Rot(Delta_j) Rot(omega_j) (scipy); the
    root keeps omega_0."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    s = synth.subject(5)
    aa, rt = synth.random_pose(np.random.default_rng(6))
    delta = np.random.default_rng(10).normal(scale=0.2, size=(23, 3))
    layers = _layers(8)
    layers[-1] = (torch.zeros_like(layers[-1][0]), torch.from_numpy(delta.reshape(-1)))
    _, _, om = refine.refined_pose(s["parents"], s["rest_joints"], aa, rt, layers)
    ref = np.asarray(aa, np.float64).copy()
    ref[1:] = (Rot.from_rotvec(delta) * Rot.from_rotvec(ref[1:])).as_rotvec()
    assert np.allclose(om.numpy().reshape(-1, 3), ref, atol=1e-12)


def test_without_refiner_is_the_numpy_fk():
    s = synth.subject(3)
    aa, rt = synth.random_pose(np.random.default_rng(4))
    R, t = refine.refined_transforms(s["parents"], s["rest_joints"], aa, rt, None)
    R0, t0 = fk.bone_transforms(s["parents"], s["rest_joints"], aa, rt)
    assert np.allclose(R.numpy(), R0, atol=1e-14) and np.allclose(t.numpy(), t0, atol=1e-14)


def test_fixed_correction_composes_rotations():
    """Output layer W = 0, b = Delta: the refined pose has local rotations Rot(Delta_j) Rot(omega_j),
    i.e. the numpy FK of the composed axis-angles (composition by scipy)."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    s = synth.subject(5)
    aa, rt = synth.random_pose(np.random.default_rng(6))
    rng = np.random.default_rng(7)
    delta = rng.normal(scale=0.2, size=(23, 3))
    layers = _layers(8)
    W, b = layers[-1]
    layers[-1] = (torch.zeros_like(W), torch.from_numpy(delta.reshape(-1)))
    R, t = refine.refined_transforms(s["parents"], s["rest_joints"], aa, rt, layers)
    comp = np.array(aa, np.float64).copy()
    comp[1:] = (Rot.from_rotvec(delta) * Rot.from_rotvec(np.asarray(aa, np.float64)[1:])).as_rotvec()
    R0, t0 = fk.bone_transforms(s["parents"], s["rest_joints"], comp, rt)
    assert np.allclose(R.numpy(), R0, atol=1e-12) and np.allclose(t.numpy(), t0, atol=1e-12)


def test_loss_gradient_in_refiner_weights_matches_central_differences():
    subj = synth.subject(21, hash_scale=0.5, res_last_std=0.02)
    frames = synth.training_frames(22, 2, res=32)
    for c in frames["cameras"]:
        c.n_samples = 16
    batch = synth.pixel_batch(23, 48, 2, 32, 32)
    tgt = np.random.default_rng(24).uniform(0, 1, size=(48, 3)).astype(np.float32)
    P = OF.Params(subj)
    layers = [(W.requires_grad_(True), b.requires_grad_(True)) for W, b in _layers(25)]
    loss, _ = OR.train_loss(subj, P, frames, batch, tgt, 99, 16, np.zeros(3), refiner=layers)
    loss.backward()

    def f():
        with torch.no_grad():
            return OR.train_loss(subj, P, frames, batch, tgt, 99, 16, np.zeros(3), refiner=layers)[0].item()

    rng = np.random.default_rng(0)
    checked = skipped = 0
    for ten in (layers[0][0], layers[1][0], layers[-1][0], layers[-1][1]):
        g = ten.grad.reshape(-1)
        nz = torch.nonzero(g.abs() > 1e-9).squeeze(1).numpy()
        for j in rng.choice(nz, size=min(12, len(nz)), replace=False):
            flat = ten.data.reshape(-1)
            old = flat[j].item()
            fds = []
            for e in (1e-5, 1e-6):
                flat[j] = old + e
                lp = f()
                flat[j] = old - e
                lm = f()
                flat[j] = old
                fds.append((lp - lm) / (2 * e))
            if abs(fds[0] - fds[1]) > 1e-6 * max(1e-3, abs(fds[0])):
                skipped += 1
                continue
            assert abs(fds[0] - g[j].item()) <= 1e-5 * max(1e-3, abs(fds[0])) + 1e-10
            checked += 1
    assert checked >= 16 and skipped <= 2 * checked, (checked, skipped)
