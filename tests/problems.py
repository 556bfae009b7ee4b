"""Shared test fixtures: seeded workloads with oracle-made data (tests only)."""
from __future__ import annotations

import functools

import numpy as np

import synthetic as S
from oracle import fem, rto, wave


@functools.lru_cache(maxsize=8)
def cube_problem(n, n_obs, n_steps, faces=S.ALL_FACES, seed=1, dt_factor=0.3, phantom="blobs3", noise=0.01,
                 data=False):
    """Mesh, oracle operators and p0 of a Kuhn cube; with ``data`` also the noisy
    observations y_obs = G p0 + eta (oracle forward, eq. noise-model) and sigma."""
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, faces, seed)
    p0 = S.phantom(xyz, phantom, seed + 100, n)
    ops = fem.build(xyz, tets, det, n)
    dt = dt_factor / n
    P = {"n": n, "xyz": xyz, "tets": tets, "det": det, "p0": p0, "ops": ops, "dt": dt, "n_steps": n_steps}
    if data:
        Y = wave.forward(ops, p0, dt, n_steps)
        y_obs, sigma = rto.add_noise(Y, S.standard_normal(Y.shape, seed + 2), noise, dt)
        P.update(Y=Y, y_obs=y_obs, sigma=sigma)
    return P


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def as_precision(a, prec):
    """Round an input to the GPU's state precision (both sides then see the same numbers)."""
    return np.asarray(a, dtype=np.float32 if prec == "f32" else np.float64).astype(np.float64)
