"""Seeded input generators (host logic, no GPU): the batch layouts the training
step consumes."""
import numpy as np

from paper_2306_16541_gb300 import synth


def test_patch_batch_layout():
    """Sec. 5.2: each drawn image contributes 6 square 20 x 20 patches, in bounds."""
    b = synth.patch_batch(5, frames=7, n_images=3, width=64, height=48)
    fr, px, py = b["frame"], b["px"], b["py"]
    assert fr.shape == px.shape == py.shape == (3 * 6 * 400,)
    assert fr.dtype == px.dtype == py.dtype == np.uint32
    assert fr.max() < 7 and px.max() < 64 and py.max() < 48
    for p in range(18):
        sl = slice(p * 400, (p + 1) * 400)
        assert len(set(fr[sl].tolist())) == 1
        x, y = px[sl].astype(int), py[sl].astype(int)
        assert x.max() - x.min() == 19 and y.max() - y.min() == 19
        assert len(set(zip(x.tolist(), y.tolist()))) == 400
    again = synth.patch_batch(5, frames=7, n_images=3, width=64, height=48)
    assert all(np.array_equal(b[k], again[k]) for k in b)


def test_pixel_batch_in_bounds():
    b = synth.pixel_batch(9, 1000, 5, 40, 30)
    assert b["frame"].max() < 5 and b["px"].max() < 40 and b["py"].max() < 30
