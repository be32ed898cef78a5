"""Adam update (oracle, FP64).  Test infrastructure only.

Sec. 5.2 trains with Adam, beta1 = 0.9, beta2 = 0.99.  One step on parameter
p with gradient g, moments m and v and step count k (1-based), with bias
correction as in Kingma and Ba (2015):
    m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2
    p <- p - lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps)
Every entry is updated, including those whose gradient is zero.
"""
from __future__ import annotations

import numpy as np


def adam_step(p, g, m, v, k: int, lr: float, b1: float = 0.9, b2: float = 0.99, eps: float = 1e-8):
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
