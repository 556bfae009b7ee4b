"""P1 finite-element matrices and sensor interpolation (oracle, FP64).

Section 3 of the paper: with piecewise-linear basis functions phi_i,
  M_mn = int phi_m phi_n dx,  K_mn = c^2 int grad phi_m . grad phi_n dx,
  B_mn = (1/c) int_{boundary} phi_m phi_n ds            (eq. semi-discrete)
and the lumped mass M_L = diag(M 1) (mass lumping paragraph after
eq. fully-discrete).  B is assembled at c = 1 (the paper's nondimensional
setting); a per-element c^2 enters K only.

Sensors (Section 3, eq. lagrange, and the remark in Section 5.1 that Pi^T is the
transpose of an interpolation operator when sensors are not nodes): a sensor at
a boundary point is interpolated with the P1 basis of the boundary triangle
holding it.  On the structured Kuhn cube this triangle is found from the face
lattice directly (no geometric search), which is independent of how the CUDA
library locates sensors.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def element_geometry(xyz, tets):
    """Volumes and barycentric gradients of every tetrahedron.

    For vertices X0..X3 let J = [X1-X0, X2-X0, X3-X0]; the barycentric
    coordinates are lambda_{1..3} = J^{-1} (x - X0), lambda_0 = 1 - sum, so
    grad lambda_a is row a of J^{-1} and grad lambda_0 = -(sum of rows).
    Returns vol (E,) and grads (E, 4, 3).
    """
    X = xyz[tets]                                    # (E, 4, 3)
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    det = np.linalg.det(J)
    vol = np.abs(det) / 6.0
    Jinv = np.linalg.inv(J)                          # rows = grad lambda_1..3
    grads = np.empty((len(tets), 4, 3))
    grads[:, 1:, :] = Jinv
    grads[:, 0, :] = -Jinv.sum(axis=1)
    return vol, grads


def assemble(xyz, tets, c2_elem=None):
    """Assemble M (consistent), M_L, K and B as SciPy CSR matrices.

    Consistent P1 tetrahedron mass: M_e = V/20 (1 + delta_ab).
    Stiffness: K_e = c_e^2 V grad(lambda_a) . grad(lambda_b).
    Boundary faces are triangles that belong to exactly one tetrahedron;
    consistent P1 triangle mass B_f = A/12 (1 + delta_ab).
    Returns a dict with M, ML (vector), K, B, bfaces (F, 3), vol, grads.
    """
    N = len(xyz)
    E = len(tets)
    vol, grads = element_geometry(xyz, tets)
    c2 = np.ones(E) if c2_elem is None else np.asarray(c2_elem, dtype=np.float64)

    rows = np.repeat(tets, 4, axis=1).ravel()        # (E*16,) a-index
    cols = np.tile(tets, (1, 4)).ravel()             # b-index
    Me = (vol[:, None, None] / 20.0) * (np.ones((4, 4)) + np.eye(4))
    Ke = (c2 * vol)[:, None, None] * np.einsum("eai,ebi->eab", grads, grads)
    M = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(N, N))
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(N, N))
    ML = np.asarray(M.sum(axis=1)).ravel()           # M_L = diag(M 1)

    # boundary faces: the 4 faces of each tet, kept when seen exactly once
    faces = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]],
                            tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]])
    key = np.sort(faces, axis=1)
    uniq, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    bfaces = uniq[cnt == 1]
    P = xyz[bfaces]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    Be = (area[:, None, None] / 12.0) * (np.ones((3, 3)) + np.eye(3))
    brows = np.repeat(bfaces, 3, axis=1).ravel()
    bcols = np.tile(bfaces, (1, 3)).ravel()
    B = sp.csr_matrix((Be.ravel(), (brows, bcols)), shape=(N, N))
    return {"M": M, "ML": ML, "K": K, "B": B, "bfaces": bfaces, "vol": vol, "grads": grads,
            "c2": c2}


def sensor_weights_cube(n, det_xyz):
    """P1 interpolation of sensors on the faces of the Kuhn cube.

    A point on face (axis fixed at 0 or 1) has in-plane coordinates (u, v) in
    increasing axis order.  With i = min(floor(u n), n-1), j likewise, and
    fu = u n - i, fv = v n - j, the face square's diagonal runs from its low
    corner v00 to its high corner v11 (every Kuhn edge increases all changed
    coordinates), so the holding triangle and its P1 weights are
      fu >= fv:  (v00, v10, v11) with (1 - fu, fu - fv, fv)
      fu <  fv:  (v00, v01, v11) with (1 - fv, fv - fu, fu).
    Returns nodes (N_obs, 3) int64 and weights (N_obs, 3) float64.
    """
    det_xyz = np.asarray(det_xyz, dtype=np.float64)
    nodes = np.empty((len(det_xyz), 3), dtype=np.int64)
    w = np.empty((len(det_xyz), 3))
    for d, x in enumerate(det_xyz):
        on = [a for a in range(3) if x[a] == 0.0 or x[a] == 1.0]
        if not on:
            raise ValueError(f"sensor {d} is not on the cube boundary")
        axis = on[0]
        others = [a for a in range(3) if a != axis]
        u, v = x[others[0]] * n, x[others[1]] * n
        i, j = min(int(np.floor(u)), n - 1), min(int(np.floor(v)), n - 1)
        fu, fv = u - i, v - j

        def node(du, dv):
            ijk = [0, 0, 0]
            ijk[axis] = int(round(x[axis] * n))
            ijk[others[0]] = i + du
            ijk[others[1]] = j + dv
            return (ijk[0] * (n + 1) + ijk[1]) * (n + 1) + ijk[2]

        if fu >= fv:
            nodes[d] = (node(0, 0), node(1, 0), node(1, 1))
            w[d] = (1.0 - fu, fu - fv, fv)
        else:
            nodes[d] = (node(0, 0), node(0, 1), node(1, 1))
            w[d] = (1.0 - fv, fv - fu, fu)
    return nodes, w


def sensor_weights_nodes(xyz, det_xyz):
    """Node-coincident sensors: each sensor position equals a mesh node's
    coordinates (to 1e-12 of the mesh size); its observation is that node's
    value.  Returns nodes (N_obs, 1) int64 and weights (N_obs, 1)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    det_xyz = np.asarray(det_xyz, dtype=np.float64)
    scale = np.ptp(xyz, axis=0).max()
    nodes = np.empty((len(det_xyz), 1), dtype=np.int64)
    for d, x in enumerate(det_xyz):
        dist = np.abs(xyz - x).max(axis=1)
        i = int(np.argmin(dist))
        if dist[i] > 1e-12 * scale:
            raise ValueError(f"sensor {d} does not coincide with a node")
        nodes[d, 0] = i
    return nodes, np.ones((len(det_xyz), 1))


def observation_matrix(N, nodes, weights):
    """Pi as a sparse (N_obs, N) matrix: row d holds the sensor's P1 weights."""
    n_obs = len(nodes)
    rows = np.repeat(np.arange(n_obs), nodes.shape[1])
    return sp.csr_matrix((weights.ravel(), (rows, nodes.ravel())), shape=(n_obs, N))


def sensor_weights_points(xyz, tets, det_xyz):
    """Sensors anywhere in a tetrahedral mesh, by brute force (small meshes): the
    tetrahedron that holds the point and its barycentric coordinates, i.e. the
    P1 interpolation weights of its four vertices (eq. lagrange).  A point on a
    shared face or edge takes the holding tetrahedron of smallest index."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    P0 = xyz[tets[:, 0]]
    J = np.stack([xyz[tets[:, v]] - P0 for v in (1, 2, 3)], axis=2)     # (E, 3, 3), edges as columns
    Jinv = np.linalg.inv(J)
    nodes = np.empty((len(det_xyz), 4), dtype=np.int64)
    w = np.empty((len(det_xyz), 4))
    for d, x in enumerate(np.asarray(det_xyz, dtype=np.float64)):
        l123 = np.einsum("eij,ej->ei", Jinv, x - P0)
        lam = np.concatenate([1.0 - l123.sum(axis=1)[:, None], l123], axis=1)
        inside = np.nonzero(lam.min(axis=1) >= -1e-12)[0]
        if len(inside) == 0:
            raise ValueError(f"sensor {d} is outside the mesh")
        e = inside[0]
        lm = np.maximum(lam[e], 0.0)
        nodes[d] = tets[e]
        w[d] = lm / lm.sum()
    return nodes, w


def build_point_sensors(xyz, tets, det_xyz, c2_elem=None):
    """All oracle operators for any tetrahedral mesh with sensors anywhere inside it."""
    ops = assemble(xyz, tets, c2_elem)
    nodes, w = sensor_weights_points(xyz, tets, det_xyz)
    ops["det_nodes"] = nodes
    ops["det_w"] = w
    ops["Pi"] = observation_matrix(len(xyz), nodes, w)
    return ops


def build_node_sensors(xyz, tets, det_xyz, c2_elem=None):
    """All oracle operators for any tetrahedral mesh with node-coincident sensors."""
    ops = assemble(xyz, tets, c2_elem)
    nodes, w = sensor_weights_nodes(xyz, det_xyz)
    ops["det_nodes"] = nodes
    ops["det_w"] = w
    ops["Pi"] = observation_matrix(len(xyz), nodes, w)
    return ops


def build(xyz, tets, det_xyz, n, c2_elem=None):
    """All oracle operators for a Kuhn cube with n^3 cells."""
    ops = assemble(xyz, tets, c2_elem)
    nodes, w = sensor_weights_cube(n, det_xyz)
    ops["det_nodes"] = nodes
    ops["det_w"] = w
    ops["Pi"] = observation_matrix(len(xyz), nodes, w)
    return ops
