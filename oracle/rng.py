"""Counter-based N(0,1) draws, restated from their published definitions (oracle).

SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): the generator seeded with s returns, as its
i-th output (i = 1, 2, ...), the mix function applied to s + i * GAMMA with
GAMMA = 0x9E3779B97F4A7C15, where mix(z) = z3 with
    z1 = (z  ^ (z  >> 30)) * 0xBF58476D1CE4E5B9
    z2 = (z1 ^ (z1 >> 27)) * 0x94D049BB133111EB
    z3 =  z2 ^ (z2 >> 31)          (all mod 2^64).
Box-Muller (1958), cosine branch: z = sqrt(-2 ln u1) cos(2 pi u2).

A draw keyed by (seed, stream, sample k, element e) uses outputs 2c+1 and 2c+2
with c = ((k << 1 | stream) << 40) | e; u1 = ((out >> 11) + 1) 2^-53 lies in
(0, 1], u2 = (out >> 11) 2^-53 in [0, 1).  The sampler does not fix a generator
(the paper draws eta and xi without saying how); this one lets a sample's draws
depend only on (seed, k), whatever the batch size.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_output(seed, i):
    """i-th output (uint64 array) of SplitMix64 seeded with ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.asarray(i, dtype=np.uint64) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def normals(seed, stream, n_elem, K, samples=None):
    """Draws for elements e < n_elem and samples k < K, shape (n_elem, K); or,
    with ``samples`` (a list of sample indices), only those columns."""
    e = np.arange(n_elem, dtype=np.uint64)[:, None]
    ks = np.arange(K) if samples is None else np.asarray(samples)
    k = ks.astype(np.uint64)[None, :]
    c = (((k << np.uint64(1)) | np.uint64(stream)) << np.uint64(40)) | e
    with np.errstate(over="ignore"):
        h1 = splitmix64_output(seed, np.uint64(2) * c + np.uint64(1))
        h2 = splitmix64_output(seed, np.uint64(2) * c + np.uint64(2))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
