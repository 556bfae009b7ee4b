"""Pins of the oracle's P1 assembly and sensor interpolation (CPU only).

Everything here is checked against closed forms of the Kuhn cube (golden file,
derived by hand from the definitions of Section 3) or against an independent
brute-force evaluation, never against the oracle itself.
"""
import json
import os

import numpy as np
import pytest

import synthetic as S
from oracle import fem

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "kuhn_cube_closed_forms.json")))


@pytest.fixture(scope="module", params=[3, 6])
def cube(request):
    n = request.param
    xyz, tets = S.cube_mesh(n)
    return n, xyz, tets, fem.assemble(xyz, tets)


def test_mesh_numbering():
    xyz, tets = S.cube_mesh(2)
    assert xyz.shape == (27, 3) and tets.shape == (48, 4)
    # first cell, first permutation (x, y, z): path 0 -> +x -> +x+y -> +x+y+z
    assert tets[0].tolist() == [0, 9, 12, 13]
    # every tet has positive volume h^3 / 6
    X = xyz[tets]
    vol = np.abs(np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], 2))) / 6
    assert np.allclose(vol, (0.5 ** 3) / 6, rtol=0, atol=1e-15)


def test_global_sums(cube):
    n, xyz, tets, ops = cube
    assert abs(ops["ML"].sum() - GOLD["domain_volume"]) < 1e-13
    assert abs(ops["B"].sum() - GOLD["boundary_area"]) < 1e-12
    assert np.abs(ops["K"] @ np.ones(len(xyz))).max() < 1e-13       # constants are in K's kernel
    assert abs(ops["M"].sum() - 1.0) < 1e-13
    for A in (ops["K"], ops["B"], ops["M"]):
        assert abs(A - A.T).max() < 1e-15


def test_interior_row_is_seven_point_laplacian(cube):
    n, xyz, tets, ops = cube
    h = 1.0 / n
    g = GOLD["interior_K_row_over_h"]
    K = ops["K"].tocsr()
    for (i, j, k) in [(1, 1, 1), (n // 2, n // 2, n - 1 if n > 2 else 1)]:
        row = S.node_index(i, j, k, n)
        cols = K.indices[K.indptr[row]:K.indptr[row + 1]]
        vals = K.data[K.indptr[row]:K.indptr[row + 1]] / h
        assert len(cols) == GOLD["kuhn_graph_entries_per_interior_row"]
        axis = {S.node_index(i + a, j + b, k + c, n) for a, b, c in
                [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]}
        for c, v in zip(cols, vals):
            if c == row:
                assert abs(v - g["diagonal"]) < 1e-12
            elif c in axis:
                assert abs(v - g["axis_neighbours"]) < 1e-12
            else:
                assert abs(v - g["other_graph_entries"]) < 1e-12
        assert abs(ops["ML"][row] / h ** 3 - GOLD["interior_ML_over_h3"]) < 1e-12


def test_corner_masses_and_boundary_rows(cube):
    n, xyz, tets, ops = cube
    h = 1.0 / n
    c = GOLD["corner_ML_over_h3"]
    for (i, j, k) in [(0, 0, 0), (n, n, n)]:
        assert abs(ops["ML"][S.node_index(i, j, k, n)] / h ** 3 - c["main_diagonal_corners"]) < 1e-12
    for (i, j, k) in [(n, 0, 0), (0, n, 0), (0, 0, n), (n, n, 0), (n, 0, n), (0, n, n)]:
        assert abs(ops["ML"][S.node_index(i, j, k, n)] / h ** 3 - c["other_corners"]) < 1e-12
    rs = np.asarray(ops["B"].sum(axis=1)).ravel()
    row = S.node_index(0, 1, 1, n)        # interior of face x = 0
    assert abs(rs[row] / h ** 2 - GOLD["face_interior_B_rowsum_over_h2"]) < 1e-12
    # B touches boundary nodes only
    on_bnd = np.any((xyz == 0.0) | (xyz == 1.0), axis=1)
    assert np.all(rs[~on_bnd] == 0.0) and np.all(rs[on_bnd] > 0.0)
    assert len(ops["bfaces"]) == 12 * n * n


def brute_force_sensor(xyz, bfaces, x):
    """Independent location: the boundary triangle whose barycentrics are all >= 0."""
    best = None
    for f in bfaces:
        P = xyz[f]
        e1, e2 = P[1] - P[0], P[2] - P[0]
        nrm = np.cross(e1, e2)
        if abs(np.dot(x - P[0], nrm)) > 1e-12:
            continue
        G = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
        b = np.linalg.solve(G, [e1 @ (x - P[0]), e2 @ (x - P[0])])
        lam = np.array([1 - b.sum(), b[0], b[1]])
        if lam.min() >= -1e-12 and (best is None or lam.min() > best[1].min()):
            best = (f, lam)
    return best


@pytest.mark.parametrize("n", [3, 8])
def test_sensor_interpolation(n):
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(40, S.ALL_FACES, 7)
    ops = fem.assemble(xyz, tets)
    nodes, w = fem.sensor_weights_cube(n, det)
    bf = {tuple(sorted(f)) for f in ops["bfaces"].tolist()}
    assert np.all(w >= 0) and np.allclose(w.sum(1), 1.0, atol=1e-15)
    for d in range(len(det)):
        assert tuple(sorted(nodes[d].tolist())) in bf
    # P1 interpolation reproduces linear functions exactly
    f = lambda X: 0.3 + 1.7 * X[..., 0] - 0.9 * X[..., 1] + 2.3 * X[..., 2]
    Pi = fem.observation_matrix(len(xyz), nodes, w)
    assert np.abs(Pi @ f(xyz) - f(det)).max() < 1e-13
    # the same triangle and weights as a brute-force geometric search
    for d in range(len(det)):
        f_bf, lam = brute_force_sensor(xyz, ops["bfaces"], det[d])
        a = dict(zip(nodes[d].tolist(), w[d]))
        b = dict(zip(f_bf.tolist(), lam))
        keys = {k for k in set(a) | set(b) if max(a.get(k, 0), b.get(k, 0)) > 1e-12}
        for k in keys:
            assert abs(a.get(k, 0.0) - b.get(k, 0.0)) < 1e-12


# ---------------------------------------------------------------------------
# A non-cube mesh: the ball carved from the Kuhn mesh, node-coincident sensors
# ---------------------------------------------------------------------------
def _boundary_faces_independent(tets):
    """Faces belonging to exactly one tetrahedron, found by counting sorted triples."""
    faces = np.sort(np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]], tets[:, [0, 2, 3]],
                                    tets[:, [1, 2, 3]]]), axis=1)
    uniq, cnt = np.unique(faces, axis=0, return_counts=True)
    return uniq[cnt == 1]


def test_carved_sphere_operators_have_their_closed_form_sums():
    """Every Kuhn tetrahedron of cell size h has volume h^3/6, so sum M_L = E h^3/6;
    K annihilates constants; 1^T B 1 is the boundary area (B_f = A_f/12 (1 + delta_ab))."""
    n, R = 10, 2.0
    xyz, tets = S.sphere_mesh(n, R)
    h = 2 * R / n
    ops = fem.assemble(xyz, tets)
    assert abs(ops["ML"].sum() - len(tets) * h ** 3 / 6) <= 1e-12 * len(tets) * h ** 3
    assert np.abs(ops["K"] @ np.ones(len(xyz))).max() <= 1e-13 * np.abs(ops["K"]).max()
    bf = _boundary_faces_independent(tets)
    P = xyz[bf]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1).sum()
    one = np.ones(len(xyz))
    assert abs(one @ (ops["B"] @ one) - area) <= 1e-12 * area
    assert 4 * np.pi * R * R < area < 4 * np.pi * R * R * 2.0       # a stair-cased sphere: larger than 4 pi R^2
    r = np.linalg.norm(xyz, axis=1)
    assert r.max() <= R + np.sqrt(3) * h and len(np.unique(tets)) == len(xyz)


def test_node_sensors_observe_the_node_values():
    n, R = 10, 2.0
    xyz, tets = S.sphere_mesh(n, R)
    det = S.octant_node_sensors(xyz, 12, 1.0, 2 * R / n, 5)
    ops = fem.build_node_sensors(xyz, tets, det)
    f = xyz @ np.array([0.3, -1.2, 0.7]) + 0.25                 # any nodal field
    assert np.abs(ops["Pi"] @ f - (det @ np.array([0.3, -1.2, 0.7]) + 0.25)).max() < 1e-14
    assert np.all(det >= 0.0) and np.all(np.abs(np.linalg.norm(det, axis=1) - 1.0) <= R / n)


def test_point_sensors_interpolate_linear_fields_exactly():
    """P1 interpolation inside a tetrahedron reproduces linear fields (eq. lagrange),
    and the weights are a partition of unity over the holding tetrahedron."""
    xyz, tets = S.sphere_mesh(8, 2.0)
    det = S.octant_sphere_points(20, 1.0, 3)
    nodes, w = fem.sensor_weights_points(xyz, tets, det)
    a, b = np.array([0.3, -1.2, 0.7]), 0.25
    f = xyz @ a + b
    assert np.abs((w * f[nodes]).sum(axis=1) - (det @ a + b)).max() < 1e-13
    assert np.all(w >= 0.0) and np.abs(w.sum(axis=1) - 1.0).max() < 1e-14
    with pytest.raises(ValueError):
        fem.sensor_weights_points(xyz, tets, np.array([[5.0, 0.0, 0.0]]))
