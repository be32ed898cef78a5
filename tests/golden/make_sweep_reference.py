"""Writes sweep_oracle_pixels.txt: the FP64 oracle's RGBA (Sec. 2.1 Eq. 3 with the field of
Sec. 4.2-4.4, no early termination, no occupancy) at the precision sweep's seeded pixels of
both sweep fields (1920x1080, 192 samples per ray), for bench.py's precision sweep, which
compares every tier with these values and does not run the oracle itself.

    python tests/golden/make_sweep_reference.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import field as OF          # noqa: E402
from oracle import render as OR         # noqa: E402
from paper_2306_16541_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "sweep_oracle_pixels.txt")


def main():
    cfg, variants = synth.sweep_variants()
    cam = cfg["camera"]
    px, py = synth.sweep_pixels(cam.width, cam.height)
    lines = ["# FP64 oracle RGBA at the precision sweep's pixels (synth.sweep_variants, synth.sweep_pixels):",
             "# 1920x1080, 192 samples per ray, no occupancy, no early termination.",
             "# Written by tests/golden/make_sweep_reference.py from oracle/ only.",
             "# columns: variant px py r g b a"]
    for name, subj in variants:
        ref = OR.render_pixels(subj, OF.Params(subj), cfg["pose"], cam, px, py, False).numpy()
        for i in range(len(px)):
            lines.append(f"{name} {int(px[i])} {int(py[i])} " + " ".join(f"{v:.17g}" for v in ref[i]))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
