"""Pins of the oracle's density-grid occupancy (Sec. 2.3 empty-space skipping
carried by the field's own density): a library dilation, a closed-form density,
an exact translation of the grid, and the bit layout the marcher reads."""
import numpy as np
import pytest
import torch

from oracle import decide32, fk
from oracle import field as OF
from oracle import occupancy as OO
from paper_2306_16541_gb300 import synth


@pytest.mark.parametrize("r", [0, 1, 2])
def test_dilation_matches_scipy(r):
    ndimage = pytest.importorskip("scipy.ndimage")
    g = 12
    m = np.random.default_rng(r).uniform(size=g ** 3) < 0.03
    ref = ndimage.binary_dilation(m.reshape(g, g, g), structure=np.ones((2 * r + 1,) * 3, bool), border_value=0)
    assert np.array_equal(OO.dilate(m, g, r), ref.reshape(-1))


def test_pack_matches_marcher_bit_layout():
    g = 16
    m = np.random.default_rng(3).uniform(size=g ** 3) < 0.4
    words = OO.pack(m)
    assert words.shape == (g ** 3 // 32,) and words.dtype == np.uint32
    assert np.array_equal(decide32.bit_test(words, np.arange(g ** 3)), m)
    assert np.array_equal(OO.unpack(words), m)


def _linear_density_subject(a, c, seed=5):
    """Shaped-density subject whose density feature is the linear function a . v + c on its
    dense level: the encoding reproduces it exactly, so sigma = softplus(beta (a . y + c) + bias)."""
    s = synth.shaped_density(synth.subject(seed, with_ellipsoids=True, hash_scale=0.5), beta=3.0, bias=-1.0)
    levels = [int(n) for n in s["level_res"]]
    T = 1 << int(s["log2_T"])
    lv = [l for l, n in enumerate(levels) if (n + 1) ** 3 <= T][-1]
    n = levels[lv]
    iz, iy, ix = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    v = -1.0 + 2.0 * np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1) / n
    tab = s["hash_table"].copy()
    tab[lv, ix.ravel() + iy.ravel() * (n + 1) + iz.ravel() * (n + 1) ** 2, 0] = (v @ a + c).astype(np.float32)
    s["hash_table"] = tab
    return s


def test_canonical_density_closed_form():
    a, c = np.array([0.25, -0.5, 0.75]), 0.125
    s = _linear_density_subject(a, c)
    g = 16
    sigma = OO.canonical_sigma(OF.Params(s), g).numpy()
    j = (np.arange(g) + 0.5) / g * 2.0 - 1.0
    z, y, x = np.meshgrid(j, j, j, indexing="ij")
    o3 = 3.0 * (a[0] * x + a[1] * y + a[2] * z + c).ravel() - 1.0
    # the table stores a . v + c rounded to float32 (vertices at multiples of 2 / 23)
    assert np.allclose(sigma, np.logaddexp(0.0, o3), rtol=0, atol=1e-6)
    canon, _ = OO.canonical_grid(OF.Params(s), g, 0.5, 0)
    ref = np.logaddexp(0.0, o3)
    far = np.abs(ref - 0.5) > 1e-5
    assert far.sum() > 0.9 * g ** 3
    assert np.array_equal(canon[far], (ref > 0.5)[far]) and 0 < canon.sum() < g ** 3


def test_posed_grid_of_a_translation_is_a_shifted_grid():
    """Uniform weights (S = 1 inside the box), no residual, root moved by k whole cells
    along x: G_i(y) = y - t, so posed(c) = canon(c - k e_x), empty where c_x < k."""
    g, k = 16, 3
    s = synth.subject(7)
    s["wvol"] = np.full_like(s["wvol"], 1.0 / 24.0)
    s["wvol"][24] = 0.0
    s["res_enabled"] = 0
    P = OF.Params(s)
    h = 2.0 / g
    aa = np.zeros((24, 3), np.float32)
    rt = np.array([k * h, 0.0, 0.0], np.float32)
    R, t = fk.bone_transforms(s["parents"], s["rest_joints"], aa, rt)
    assert np.allclose(R, np.eye(3)[None], atol=1e-15) and np.allclose(t, -rt[None].astype(np.float64), atol=1e-12)
    canon = np.random.default_rng(11).uniform(size=g ** 3) < 0.3
    S, xf = OO.posed_points(P, torch.from_numpy(R), torch.from_numpy(t), torch.zeros(72, dtype=torch.float64), g)
    posed = OO.posed_grid(canon, S, xf, s["box_min"], s["box_max"], g, 0.5)
    ref = np.zeros((g, g, g), bool)
    ref[:, :, k:] = canon.reshape(g, g, g)[:, :, :g - k]
    assert np.array_equal(posed.reshape(g, g, g), ref)
