"""C-ABI checks that need no GPU: exported symbols and the host-side assembly.

The library's FP64 host assembly (pat_mesh_create with PAT_MESH_HOST_ONLY) is
compared with the oracle's independent assembly: connectivity and sensor
triangles bit-exact, values to FP64 rounding.
"""
import os
import re
import subprocess

import numpy as np
import pytest

import synthetic as S
from oracle import fem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pat.h")).read()
    return sorted(set(re.findall(r"^\s*(?:pat_status|const char\*)\s+(pat_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_21373_b300 import _lib
    return _lib.load()


def test_library_exports_every_declared_symbol(lib):
    from paper_2607_21373_b300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pat_\w+)", out))
    decl = declared_symbols()
    assert len(decl) >= 15
    missing = [s for s in decl if s not in exported]
    assert not missing, missing
    from paper_2607_21373_b300 import _lib
    assert set(decl) <= set(_lib.SIGNATURES)


def host_mesh(n, n_obs, faces, seed, dt_factor=0.3, flags=0x8 | 0x1):
    from paper_2607_21373_b300 import Mesh
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, faces, seed)
    m = Mesh(xyz, tets, det, dt_factor / n, 10, precision="f64", flags=flags)
    return m, xyz, tets, det


@pytest.mark.parametrize("n", [3, 8])
def test_host_assembly_matches_oracle(n):
    m, xyz, tets, det = host_mesh(n, 40, S.ALL_FACES, 3)
    ops = fem.build(xyz, tets, det, n)
    ex = m.export()
    assert np.abs(ex["ML"] - ops["ML"]).max() < 1e-15
    for which, A in ((0, ops["K"]), (1, ops["B"])):
        rp, col, val = m.export_csr(which)
        A = A.tocsr()
        A.sort_indices()
        assert np.array_equal(rp, A.indptr) and np.array_equal(col, A.indices)
        assert np.abs(val - A.data).max() < 1e-14 * np.abs(A.data).max()
    bf = np.sort(ops["bfaces"], axis=1)
    bf = bf[np.lexsort(bf.T[::-1])]
    assert np.array_equal(ex["bfaces"], bf)
    # sensors: the (node -> weight) map is unique; nodes bit-exact where the weight is not ~0
    for d in range(len(det)):
        a = {int(k): w for k, w in zip(ex["det_nodes"][d], ex["det_w"][d]) if w > 1e-12}
        b = {int(k): w for k, w in zip(ops["det_nodes"][d], ops["det_w"][d]) if w > 1e-12}
        assert set(a) == set(b)
        for k in a:
            assert abs(a[k] - b[k]) < 1e-13
    info = m.info
    assert info["nnz_K_graph"] == ops["K"].nnz
    rp, col, val = m.export_csr(0)
    assert info["nnz_K"] == np.count_nonzero(val)     # the device drops entries that assembled to 0.0
    assert np.all(np.abs(ops["K"].data[np.abs(ops["K"].data) < 1e-14]) < 1e-16)
    assert info["n_boundary_faces"] == 12 * n * n


def test_unstable_time_step_is_refused():
    from paper_2607_21373_b300 import PatError
    with pytest.raises(PatError, match="PAT_EUNSTABLE"):
        host_mesh(8, 32, S.ALL_FACES, 1, dt_factor=0.4, flags=0x8)
    host_mesh(8, 32, S.ALL_FACES, 1, dt_factor=0.3, flags=0x8)   # stable: no error


def test_bad_inputs_are_rejected():
    from paper_2607_21373_b300 import Mesh, PatError
    xyz, tets = S.cube_mesh(2)
    det = S.detector_points(4, S.ALL_FACES, 1)
    with pytest.raises(PatError, match="PAT_EINVAL"):        # sensor outside the mesh
        Mesh(xyz, tets, det + np.array([0.0, 0.0, 1.5]), 0.1, 5, "f64", flags=0x8)
    # a sensor just inside the mesh is read by interpolation in its tetrahedron
    Mesh(xyz, tets, det + np.array([0.0, 0.0, 1e-3]) * (det[:, 2:3] < 1) - np.array([0.0, 0.0, 1e-3]) * (det[:, 2:3] == 1),
         0.1, 5, "f64", flags=0x8)
    bad = tets.copy()
    bad[3, 2] = 10_000
    with pytest.raises(PatError, match="PAT_EINVAL"):        # vertex index out of range
        Mesh(xyz, bad, det, 0.1, 5, "f64", flags=0x8)
    flat = tets.copy()
    flat[0] = [0, 1, 2, 2]
    with pytest.raises(PatError, match="PAT_EINVAL"):        # degenerate tetrahedron
        Mesh(xyz, flat, det, 0.1, 5, "f64", flags=0x8)
    with pytest.raises(PatError, match="PAT_EINVAL"):        # dt <= 0
        Mesh(xyz, tets, det, 0.0, 5, "f64", flags=0x8)


def test_compute_on_host_only_mesh_is_refused():
    import torch
    from paper_2607_21373_b300 import PatError, _lib
    m, *_ = host_mesh(2, 4, S.ALL_FACES, 1)
    L = _lib.load()
    import ctypes as C
    st = L.pat_forward(m._h, C.c_void_p(16), 1, C.c_void_p(16), 1.0, C.c_void_p(256), 1 << 30, None)
    assert st == 1 and b"HOST_ONLY" in L.pat_last_error()


def test_variant_selection_validates_combinations():
    """pat_select_variant is pure host logic: it accepts the documented step-kernel
    variants and refuses combinations that do not exist (PAT_EINVAL), without a GPU."""
    from paper_2607_21373_b300 import PatError
    n = 2
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(4, S.ALL_FACES, 1)
    from paper_2607_21373_b300 import Mesh
    m = Mesh(xyz, tets, det, 0.3 / n, 5, "f32", flags=0x8)
    good = [dict(V=8, packed=3, persistent=1, pdl=True, prefetch=1),
            dict(V=8, packed=3, persistent=1, pdl=True, big_blocks=True),
            dict(V=8, packed=3, persistent=3), dict(V=8, packed=3, persistent=2),
            dict(V=8, packed=3, persistent=1, gather_batch=2, min_blocks=6),
            dict(V=8, packed=3, persistent=1, gather_batch=4, min_blocks=5),
            dict(V=4, packed=1, chunk=8), dict(V=4, packed=0, staged=True), dict(V=8, packed=2)]
    for v in good:
        for d in ("fwd", "adj"):
            m.select_variant(64, d, **v)
    bad = [(64, dict(V=8, packed=1, chunk=8)),                     # chunk 8 only with V = 4
           (64, dict(V=8, packed=0)),                               # the generic kernel has no V = 8
           (64, dict(V=8, packed=3, min_blocks=6)),                 # would spill
           (64, dict(V=8, packed=3, persistent=1, min_blocks=5)),   # min_blocks 5 needs a per-batch gather
           (12, dict(V=8, packed=3)),                               # V must divide K
           (64, dict(V=4, packed=3, prefetch=9)),                   # prefetch distance 0..4
           (1, dict(V=1, packed=3, prefetch=1)),                    # no prefetch for K = 1
           (0, dict(V=1, packed=0))]                                # K out of range
    for K, v in bad:
        with pytest.raises(PatError, match="PAT_EINVAL"):
            m.select_variant(K, "fwd", **v)


def test_host_assembly_of_a_carved_sphere_with_node_sensors_matches_oracle():
    """A non-cube mesh (ball carved from the Kuhn mesh) and interior node-coincident
    sensors: the library's FP64 assembly and sensor map equal the oracle's."""
    from paper_2607_21373_b300 import Mesh
    n, R = 8, 2.0
    xyz, tets = S.sphere_mesh(n, R)
    det = S.octant_node_sensors(xyz, 10, 1.0, 2 * R / n, 7)
    m = Mesh(xyz, tets, det, 0.3 * 2 * R / n, 10, precision="f64", flags=0x8 | 0x1)
    ops = fem.build_node_sensors(xyz, tets, det)
    ex = m.export()
    assert np.abs(ex["ML"] - ops["ML"]).max() < 1e-15 * ops["ML"].max()
    for which, A in ((0, ops["K"]), (1, ops["B"])):
        rp, col, val = m.export_csr(which)
        A = A.tocsr()
        A.sort_indices()
        assert np.array_equal(rp, A.indptr) and np.array_equal(col, A.indices)
        assert np.abs(val - A.data).max() < 1e-14 * np.abs(A.data).max()
    for d in range(len(det)):
        a = {int(k): w for k, w in zip(ex["det_nodes"][d], ex["det_w"][d]) if w > 0}
        assert a == {int(ops["det_nodes"][d, 0]): 1.0}


def test_rcm_renumbering_is_a_permutation_that_narrows_the_band():
    from paper_2607_21373_b300.reorder import bandwidth, rcm_permutation, renumber
    xyz, tets = S.sphere_mesh(10, 2.0)
    N = len(xyz)
    rng = np.random.default_rng(0)
    shuffled = rng.permutation(N)
    xs, ts = renumber(xyz, tets, shuffled)
    perm = rcm_permutation(ts, N)
    assert np.array_equal(np.sort(perm), np.arange(N))
    xr, tr = renumber(xs, ts, perm)
    assert bandwidth(tr, N) < bandwidth(ts, N) / 4
    # the same mesh: every tetrahedron's vertex coordinates are unchanged
    assert np.array_equal(xr[tr], xs[ts])


def test_morton_renumbering_is_a_permutation_along_the_z_curve():
    """On the 8^3-cell cube with 16 quantisation cells per axis (lattice point
    i in cell 2i, the far face in cell 15) the Morton order starts with the 8
    corners of the first 2 x 2 x 2 cell block, x slowest, keeps the first 64
    nodes in blocks of 8 that each span one lattice cell, and keeps the mesh."""
    from paper_2607_21373_b300.reorder import morton_permutation, renumber
    xyz, tets = S.cube_mesh(8)
    perm = morton_permutation(xyz, bits=4)
    assert np.array_equal(np.sort(perm), np.arange(len(xyz)))
    xr, tr = renumber(xyz, tets, perm)
    assert np.array_equal(xr[tr], xyz[tets])
    lattice = np.rint(xr * 8).astype(int)
    assert lattice[:8].tolist() == [[0, 0, 0], [0, 0, 1], [0, 1, 0], [0, 1, 1],
                                    [1, 0, 0], [1, 0, 1], [1, 1, 0], [1, 1, 1]]
    for b in range(0, 64, 8):
        span = lattice[b:b + 8].max(axis=0) - lattice[b:b + 8].min(axis=0)
        assert np.all(span == 1)


def test_sensors_inside_tetrahedra_match_the_oracle():
    """Detectors on the physical unit sphere inside the carved ball: the library's
    holding tetrahedron and weights equal the oracle's brute-force search; a point
    outside the mesh is refused."""
    from paper_2607_21373_b300 import Mesh, PatError
    n, R = 8, 2.0
    xyz, tets = S.sphere_mesh(n, R)
    det = S.octant_sphere_points(16, 1.0, 4)
    m = Mesh(xyz, tets, det, 0.2 * 2 * R / n, 10, precision="f64", flags=0x8 | 0x1)
    nodes, w = fem.sensor_weights_points(xyz, tets, det)
    ex = m.export()
    for d in range(len(det)):
        a = {}
        for k, wt in zip(ex["det_nodes"][d], ex["det_w"][d]):
            if wt > 1e-12:
                a[int(k)] = a.get(int(k), 0.0) + wt
        b = {int(k): wt for k, wt in zip(nodes[d], w[d]) if wt > 1e-12}
        assert set(a) == set(b)
        for k in a:
            assert abs(a[k] - b[k]) < 1e-13
    with pytest.raises(PatError, match="PAT_EINVAL"):
        Mesh(xyz, tets, np.array([[5.0, 0.0, 0.0]]), 0.1, 10, precision="f64", flags=0x8 | 0x1)
