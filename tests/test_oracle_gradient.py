"""Pins of the oracle's misfit derivatives by central finite differences (CPU only)."""
import numpy as np

import synthetic as S
from oracle import fem, gradient


def test_gradients_match_finite_differences():
    n = 2
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(6, S.ALL_FACES, 3)
    rng = np.random.default_rng(1)
    c2 = (1 + 0.1 * rng.standard_normal(len(tets))) ** 2
    dt = 0.3 / n / np.sqrt(c2.max())
    ops = gradient.with_c2(fem.build(xyz, tets, det, n), tets, c2)
    p0 = rng.standard_normal(len(xyz))
    y = rng.standard_normal((30, 6))
    gp, gt = gradient.gradients(ops, tets, p0, y, dt)
    eps = 1e-6
    for e in [0, 5, 17, 47]:
        cp, cm = c2.copy(), c2.copy()
        cp[e] += eps
        cm[e] -= eps
        fd = (gradient.misfit(gradient.with_c2(ops, tets, cp), p0, y, dt)
              - gradient.misfit(gradient.with_c2(ops, tets, cm), p0, y, dt)) / (2 * eps)
        assert abs(gt[e] - fd) < 1e-6 * max(1.0, abs(fd))
    for i in [0, 3, 10, 26]:
        pp, pm = p0.copy(), p0.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (gradient.misfit(ops, pp, y, dt) - gradient.misfit(ops, pm, y, dt)) / (2 * eps)
        assert abs(gp[i] - fd) < 1e-6 * max(1.0, abs(fd))
    # directional derivative along a random theta direction
    d = rng.standard_normal(len(tets))
    fd = (gradient.misfit(gradient.with_c2(ops, tets, c2 + eps * d), p0, y, dt)
          - gradient.misfit(gradient.with_c2(ops, tets, c2 - eps * d), p0, y, dt)) / (2 * eps)
    assert abs(gt @ d - fd) < 1e-6 * abs(fd)
