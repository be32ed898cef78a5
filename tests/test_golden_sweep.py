"""The precision sweep compares every tier with stored FP64 oracle values
(tests/golden/sweep_oracle_pixels.txt, written by tests/golden/make_sweep_reference.py from
oracle/ only).  The file holds the sweep's own seeded pixels, and the oracle recomputes a
sample of its values."""
import os

import numpy as np

from oracle import field as OF
from oracle import render as OR
from paper_2306_16541_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sweep_oracle_pixels.txt")


def _stored():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            rows.setdefault(t[0], []).append([float(v) for v in t[1:]])
    return {k: np.array(v, np.float64) for k, v in rows.items()}


def test_stored_pixels_are_the_sweeps():
    cfg, variants = synth.sweep_variants()
    cam = cfg["camera"]
    px, py = synth.sweep_pixels(cam.width, cam.height)
    st = _stored()
    assert sorted(st) == sorted(name for name, _ in variants)
    for name, a in st.items():
        assert np.array_equal(a[:, 0].astype(np.int64), px)
        assert np.array_equal(a[:, 1].astype(np.int64), py)
        assert np.all(a[:, 2:] >= 0.0) and np.all(a[:, 2:] <= 1.0)


def test_oracle_reproduces_stored_values():
    cfg, variants = synth.sweep_variants()
    cam = cfg["camera"]
    st = _stored()
    pick = np.arange(0, 384, 48)
    for name, subj in variants:
        a = st[name][pick]
        ref = OR.render_pixels(subj, OF.Params(subj), cfg["pose"], cam, a[:, 0].astype(np.int64),
                               a[:, 1].astype(np.int64), False).numpy()
        # the same FP64 chain; 1e-12 leaves room for another platform's libm
        assert np.abs(ref - a[:, 2:]).max() <= 1e-12, (name, np.abs(ref - a[:, 2:]).max())
