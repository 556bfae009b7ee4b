"""The full P1 graph and unstructured-like rows on the GPU.

A P1 mesh couples each node to every node of its tetrahedra: 15 entries per
interior row.  On the regular Kuhn lattice 8 of them assemble to exactly 0.0
(the 7-point stencil remains); kept (PAT_MESH_KEEP_ZEROS) they are the rows an
unstructured mesh has, and moving the interior nodes (the jittered cube) makes
every one of them nonzero.  Such rows overflow the 8-slot fixed-width layout,
so the library builds a 16-slot copy; its kernels must give the same bits as
every other variant (same entries, same order, same arithmetic) and match the
FP64 oracle at the FP32 tolerances (1e-5 relative L2, dot test 1e-6).
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import fem, wave
from problems import as_precision, rel_l2

pytestmark = pytest.mark.gpu

WIDE_VARIANTS = [dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, early=True),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=8),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=8, early=True),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=8, early=True, min_blocks=3),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, early=True, big_blocks=True),
                 dict(V=8, packed=5, persistent=1, pdl=False, gather_batch=4),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, tail_serial=True),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, big_blocks=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, tail_serial=True, own_async=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, own_async=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True,
                      own_async=True, wide_loads=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, wide_loads=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True,
                      own_async=True, min_blocks=3),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, early=True, own_async=True),
                 dict(V=8, packed=7, persistent=1, pdl=True), dict(V=8, packed=7, persistent=1, min_blocks=3),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, own_async=True, prefetch_meta=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, prefetch_meta=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, tail_serial=True, own_async=2),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, own_async=2),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, tail_serial=True, own_async=True,
                      prefetch_meta=True),
                 dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True,
                      prefetch_meta=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, tail_serial=True, own_async=True,
                      dyn_chunks=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True,
                      dyn_chunks=True),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True,
                      own_async=3),
                 dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, own_async=3)]
# the row-quad kernel (K = 64 only: a warp is the 4 rows of a quad)
QUAD_VARIANTS = [dict(V=8, packed=8, persistent=1, pdl=True), dict(V=8, packed=8, persistent=1, pdl=True, own_async=True),
                 dict(V=8, packed=8, persistent=1, pdl=False)]
OTHER_VARIANTS = [dict(V=8, packed=3, persistent=1, pdl=True, prefetch=1), dict(V=8, packed=1, chunk=2),
                  dict(V=4, packed=0)]


def jitter_problem(n, n_obs, n_steps, seed):
    xyz, tets = S.jittered_cube_mesh(n, 0.15, seed)
    det = S.detector_points(n_obs, S.LIMITED_VIEW_FACES, seed)
    return xyz, tets, det, fem.build(xyz, tets, det, n), 0.3 / n


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("mesh_kind", ["cube_full_graph", "jitter"])
@pytest.mark.parametrize("K", [8, 24, 64, 128])
def test_wide_variants_are_bit_identical(mesh_kind, K):
    """Every variant gives the bits of the first launch, which matches the
    oracle.  1331 rows: the last 32-thread chunk is partial for every K, and
    for K = 24 (3 threads per row) chunks start and end inside rows."""
    from paper_2607_21373_b300 import MESH_KEEP_ZEROS, Mesh
    n, n_obs, nt = 10, 48, 60
    if mesh_kind == "jitter":
        xyz, tets = S.jittered_cube_mesh(n, 0.15, 11)
    else:
        xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, S.LIMITED_VIEW_FACES, 6)
    m = Mesh(xyz, tets, det, 0.3 / n, nt, precision="f32", flags=MESH_KEEP_ZEROS)
    assert m.info["nnz_K"] == m.info["nnz_K_graph"]
    p0h = as_precision(S.standard_normal((len(xyz), K), 3), "f32")
    yhh = as_precision(S.standard_normal((nt, n_obs, K), 4), "f32")
    p0, yh = dev(p0h), dev(yhh)
    Y0, g0 = m.forward(p0).clone(), m.adjoint(yh).clone()
    ops = fem.build(xyz, tets, det, n)
    assert rel_l2(Y0.cpu().numpy(), wave.forward(ops, p0h, 0.3 / n, nt)) < 1e-5
    assert rel_l2(g0.cpu().numpy(), wave.adjoint(ops, yhh, 0.3 / n)) < 1e-5
    for v in WIDE_VARIANTS + OTHER_VARIANTS + (QUAD_VARIANTS if K == 64 else []):
        if v.get("own_async") == 2 and 32 % (K // 8):
            continue  # bulk-copied own rows need whole rows per 32-thread chunk
        for d in ("fwd", "adj"):
            m.select_variant(K, d, **v)
        assert torch.equal(m.forward(p0), Y0), v
        assert torch.equal(m.adjoint(yh), g0), v


def test_sensor_terms_computed_in_the_row_where_the_buffer_does_not_fit():
    """The transposed 16-slot kernels prepare the sensor rows' terms one launch
    ahead in the fourth state buffer when 2 x (overflow entries) x K fits
    there; on a 4^3 cube with sensors on every face most nodes are sensor rows
    (each owning at least one overflow entry), so the rows compute their terms
    themselves: the same bits as the other kernels and the oracle's transpose."""
    from paper_2607_21373_b300 import MESH_KEEP_ZEROS, Mesh
    n, n_obs, nt, K = 4, 96, 30, 8
    xyz, tets = S.jittered_cube_mesh(n, 0.15, 13)
    det = S.detector_points(n_obs, S.ALL_FACES, 8)
    ops = fem.build(xyz, tets, det, n)
    m = Mesh(xyz, tets, det, 0.3 / n, nt, precision="f32", flags=MESH_KEEP_ZEROS)
    ex = m.export()
    sensor_rows = len({int(j) for row, w in zip(ex["det_nodes"], ex["det_w"]) for j, x in zip(row, w) if x > 0})
    assert 2 * sensor_rows * K + 64 > len(xyz) * K  # the inline path
    yh = as_precision(S.standard_normal((nt, n_obs, K), 9), "f32")
    m.select_variant(K, "adj", V=4, packed=0)
    g0 = m.adjoint(dev(yh)).clone()
    for v in (WIDE_VARIANTS[9], WIDE_VARIANTS[10]):
        m.select_variant(K, "adj", **v)
        assert torch.equal(m.adjoint(dev(yh)), g0), v
    assert rel_l2(g0.cpu().numpy(), wave.adjoint(ops, yh, 0.3 / n)) < 1e-5


def test_wide_single_sample_kernel_is_bit_identical():
    from paper_2607_21373_b300 import MESH_KEEP_ZEROS, Mesh
    n, n_obs, nt = 10, 48, 60
    xyz, tets = S.jittered_cube_mesh(n, 0.15, 12)
    det = S.detector_points(n_obs, S.LIMITED_VIEW_FACES, 7)
    m = Mesh(xyz, tets, det, 0.3 / n, nt, precision="f32", flags=MESH_KEEP_ZEROS)
    p0 = dev(S.standard_normal(len(xyz), 5))
    yh = dev(S.standard_normal((nt, n_obs), 6))
    Y0, g0 = m.forward(p0).clone(), m.adjoint(yh).clone()
    for v in (dict(V=1, packed=5, gather_batch=4), dict(V=1, packed=5, gather_batch=4, min_blocks=6),
              dict(V=1, packed=3), dict(V=1, packed=3, min_blocks=6), dict(V=1, packed=0)):
        for d in ("fwd", "adj"):
            m.select_variant(1, d, **v)
        assert torch.equal(m.forward(p0), Y0), v
        assert torch.equal(m.adjoint(yh), g0), v


def test_wide_variant_refused_where_it_does_not_exist():
    """16-slot rows exist for FP32 split-coefficient meshes only, with 8 samples
    per thread (K a multiple of 8) or one thread per row (K = 1)."""
    from paper_2607_21373_b300 import MESH_KEEP_ZEROS, Mesh, PatError
    xyz, tets = S.cube_mesh(6)
    det = S.detector_points(8, S.ALL_FACES, 1)
    m64 = Mesh(xyz, tets, det, 0.05, 10, precision="f64", flags=MESH_KEEP_ZEROS)
    with pytest.raises(PatError):
        m64.select_variant(8, "fwd", **WIDE_VARIANTS[0])
    m32 = Mesh(xyz, tets, det, 0.05, 10, precision="f32", flags=MESH_KEEP_ZEROS)
    with pytest.raises(PatError):
        m32.select_variant(4, "fwd", **WIDE_VARIANTS[0])
    m32.select_variant(8, "fwd", **WIDE_VARIANTS[0])


@pytest.mark.parametrize("K", [1, 16, 64])
def test_jittered_mesh_matches_oracle(K):
    """Forward, transpose and dot test on a jittered 12^3 mesh (every graph entry
    nonzero) with the 16-slot kernels (K = 64: the row-quad kernel, 2197 rows:
    a ragged last quad), against the FP64 oracle."""
    from paper_2607_21373_b300 import MESH_KEEP_ZEROS, Mesh
    n, n_obs, nt = 12, 40, 150
    xyz, tets, det, ops, dt = jitter_problem(n, n_obs, nt, 21)
    m = Mesh(xyz, tets, det, dt, nt, precision="f32", flags=MESH_KEEP_ZEROS)
    v = dict(V=1, packed=5, gather_batch=4) if K == 1 else WIDE_VARIANTS[1] if K == 16 else QUAD_VARIANTS[1]
    for d in ("fwd", "adj"):
        m.select_variant(K, d, **v)
    shape = (len(xyz),) if K == 1 else (len(xyz), K)
    p0 = as_precision(S.standard_normal(shape, 50 + K), "f32")
    yh = as_precision(S.standard_normal((nt, n_obs) + shape[1:], 51 + K), "f32")
    Y = m.forward(dev(p0))
    g = m.adjoint(dev(yh))
    assert rel_l2(Y.cpu().numpy(), wave.forward(ops, p0, dt, nt)) < 1e-5
    assert rel_l2(g.cpu().numpy(), wave.adjoint(ops, yh, dt)) < 1e-5
    lhs = float((Y.double() * dev(yh).double()).sum())
    rhs = float((dev(p0).double() * g.double()).sum())
    scale = float(Y.double().norm() * dev(yh).double().norm())
    assert abs(lhs - rhs) <= 1e-6 * scale


@pytest.mark.parametrize("mesh_kind", ["cube_full_graph", "jitter"])
def test_full_size_wide_forward_and_transpose_sampled_columns(mesh_kind):
    """The benchmark's size and launch configuration on the full graph: 205,379
    nodes, 1000 steps, 1024 sensors, K = 64, kernels chosen by the autotuner as
    bench.py does; forward and transposed solves against single-column oracle
    solves on sampled columns."""
    from paper_2607_21373_b300 import MESH_KEEP_ZEROS, Mesh
    n, n_obs, nt, seed = 58, 1024, 1000, 1003
    if mesh_kind == "jitter":
        xyz, tets = S.jittered_cube_mesh(n, 0.15, seed + 200)
    else:
        xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, S.LIMITED_VIEW_FACES, seed)
    ops = fem.build(xyz, tets, det, n)
    dt = 0.3 / n
    m = Mesh(xyz, tets, det, dt, nt, precision="f32", flags=MESH_KEEP_ZEROS)
    m.autotune(64, n_probe=10)
    p = S.phantom(xyz, "blobs20+vessels", seed + 100, n)
    rng = np.random.default_rng(1)
    p0 = as_precision(p[:, None] * rng.uniform(0.5, 1.5, size=(1, 64)), "f32")
    Y = m.forward(dev(p0))
    yh = as_precision(S.standard_normal((nt, n_obs, 64), 32), "f32")
    g = m.adjoint(dev(yh))
    for k in (0, 63):
        assert rel_l2(Y[..., k].cpu().numpy(), wave.forward(ops, p0[:, k], dt, nt)) < 1e-5
    assert rel_l2(g[:, 7].cpu().numpy(), wave.adjoint(ops, yh[..., 7], dt)) < 1e-5
