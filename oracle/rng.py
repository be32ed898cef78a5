"""SplitMix64 counter generator for stratified sample jitter (oracle side).

Test infrastructure: only tests, smoke() and the bench's CPU-baseline leg use it.

Stratified sampling (Sec. 2.1, Sec. 4.4) draws one uniform number per sample.
Both sides implement the published SplitMix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
k-th output of a generator seeded with s is mix(s + k * 0x9E3779B97F4A7C15)
with
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)
all modulo 2^64.  Sample i of batch ray r uses k = r * S + i + 1 and the
uniform u = (z >> 40) * 2^-24, which float32 holds exactly.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.asarray(k, np.uint64) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def jitter(seed: int, n_rays: int, n_samples: int, ray_offset: int = 0) -> np.ndarray:
    """u [n_rays][n_samples] in [0, 1) as float32 for batch rays ray_offset .. ray_offset+n_rays-1."""
    r = np.arange(ray_offset, ray_offset + n_rays, dtype=np.uint64)[:, None]
    i = np.arange(n_samples, dtype=np.uint64)[None, :]
    z = splitmix64(seed, r * np.uint64(n_samples) + i + np.uint64(1))
    return ((z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)
