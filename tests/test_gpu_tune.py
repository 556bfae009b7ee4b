"""Autotuning of the step kernels: every variant computes the same numbers.

Samples are independent columns and every variant walks a row's entries in the
same order, so the vector width and the shared-memory staging change where
data is read from, not the arithmetic: results must be bit-identical.
"""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K", [8, 6, 3])
def test_autotune_variants_are_bit_identical(K):
    from paper_2607_21373_b300 import Mesh
    n, n_obs, nt = 8, 32, 120
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, S.LIMITED_VIEW_FACES, 5)
    m = Mesh(xyz, tets, det, 0.3 / n, nt, precision="f32")
    p0 = torch.tensor(S.standard_normal((len(xyz), K), 1), dtype=torch.float32, device="cuda")
    yh = torch.tensor(S.standard_normal((nt, n_obs, K), 2), dtype=torch.float32, device="cuda")
    Y0, g0 = m.forward(p0).clone(), m.adjoint(yh).clone()
    table = m.autotune(K, n_probe=10)
    vs = {e["V"] for e in table}
    assert len(table) >= 2 and all(e["us_per_step"] > 0 for e in table)
    assert vs <= {v for v in (8, 4, 2, 1) if K % v == 0}
    assert torch.equal(m.forward(p0), Y0)
    assert torch.equal(m.adjoint(yh), g0)


VARIANTS = [dict(V=8, packed=2), dict(V=8, packed=1, chunk=2), dict(V=8, packed=1, chunk=4),
            dict(V=4, packed=1, chunk=4), dict(V=4, packed=1, chunk=8), dict(V=4, packed=1, chunk=2, min_blocks=6),
            dict(V=4, packed=1, chunk=4, early=True), dict(V=4, packed=0, staged=True), dict(V=4, packed=0),
            dict(V=2, packed=0), dict(V=1, packed=0), dict(V=8, packed=1, chunk=2, zorder=True),
            dict(V=4, packed=1, chunk=4, zorder=True), dict(V=8, packed=3), dict(V=4, packed=3), dict(V=8, packed=4),
            dict(V=8, packed=1, chunk=2, zorder=True, big_blocks=True), dict(V=8, packed=3, zorder=True, big_blocks=True),
            dict(V=8, packed=3, prefetch=1), dict(V=4, packed=3, prefetch=2), dict(V=8, packed=1, chunk=2, prefetch=1),
            dict(V=4, packed=3, min_blocks=6, prefetch=1), dict(V=8, packed=3, persistent=True, prefetch=1),
            dict(V=4, packed=3, persistent=True), dict(V=8, packed=3, persistent=True, zorder=True),
            dict(V=8, packed=3, persistent=True, pdl=True), dict(V=8, packed=3, persistent=True, pdl=True, prefetch=1),
            dict(V=8, packed=3, persistent=True, pdl=True, wide_loads=True),
            dict(V=8, packed=3, persistent=2, pdl=True, wide_loads=True, prefetch=1), dict(V=8, packed=3, persistent=2),
            dict(V=4, packed=3, persistent=2, prefetch=1),
            dict(V=8, packed=3, persistent=1, pdl=True, wide_loads=True, big_blocks=True),
            dict(V=8, packed=3, persistent=1, pdl=True, l2_hints=True, prefetch=1),
            dict(V=8, packed=3, persistent=3, pdl=True), dict(V=8, packed=3, persistent=3, prefetch=1),
            dict(V=8, packed=3, persistent=1, pdl=True, gather_batch=8),
            dict(V=8, packed=3, persistent=1, pdl=True, gather_batch=2, min_blocks=6),
            dict(V=8, packed=3, persistent=1, pdl=True, gather_batch=4, min_blocks=5)]


@pytest.mark.parametrize("K", [16, 64])
def test_every_variant_is_bit_identical(K):
    """Each step-kernel variant (including the tile-staged bulk-copy kernel) gives the
    same bits as the default, forward and transposed, for a whole solve."""
    from paper_2607_21373_b300 import Mesh
    n, n_obs, nt = 10, 48, 60
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, S.LIMITED_VIEW_FACES, 6)
    m = Mesh(xyz, tets, det, 0.3 / n, nt, precision="f32")
    p0 = torch.tensor(S.standard_normal((len(xyz), K), 3), dtype=torch.float32, device="cuda")
    yh = torch.tensor(S.standard_normal((nt, n_obs, K), 4), dtype=torch.float32, device="cuda")
    Y0, g0 = m.forward(p0).clone(), m.adjoint(yh).clone()
    for v in VARIANTS:
        for d in ("fwd", "adj"):
            m.select_variant(K, d, **v)
        assert torch.equal(m.forward(p0), Y0), v
        assert torch.equal(m.adjoint(yh), g0), v


def test_single_sample_variants_are_bit_identical():
    from paper_2607_21373_b300 import Mesh
    n, n_obs, nt = 10, 48, 60
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, S.LIMITED_VIEW_FACES, 7)
    m = Mesh(xyz, tets, det, 0.3 / n, nt, precision="f32")
    p0 = torch.tensor(S.standard_normal(len(xyz), 5), dtype=torch.float32, device="cuda")
    yh = torch.tensor(S.standard_normal((nt, n_obs), 6), dtype=torch.float32, device="cuda")
    Y0, g0 = m.forward(p0).clone(), m.adjoint(yh).clone()
    for v in (dict(V=1, packed=3), dict(V=1, packed=0, staged=False)):
        for d in ("fwd", "adj"):
            m.select_variant(1, d, **v)
        assert torch.equal(m.forward(p0), Y0), v
        assert torch.equal(m.adjoint(yh), g0), v
