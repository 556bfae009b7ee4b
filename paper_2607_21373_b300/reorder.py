"""Node renumbering of a tetrahedral mesh before pat_mesh_create (host, SciPy).

Reverse Cuthill-McKee (Cuthill & McKee 1969; George 1971) reduces the bandwidth
max |i - j| over the mesh's edges, which keeps a row's neighbours close in the
K-stacked fields.  A Morton (Z-order) curve through the node coordinates
(Morton 1966) instead keeps short runs of rows spatially compact in all three
directions, so the rows a thread block works on at once share more of their
neighbours.  The library accepts any numbering; observations do not depend on
it (sensors are located by position), only the fields' row order does.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

__all__ = ["node_graph", "bandwidth", "rcm_permutation", "morton_permutation", "renumber"]


def node_graph(tets, n_nodes):
    """Symmetric node adjacency (CSR, no diagonal) of the tetrahedra's edges."""
    tets = np.asarray(tets, dtype=np.int64)
    a, b = [], []
    for i in range(4):
        for j in range(4):
            if i != j:
                a.append(tets[:, i])
                b.append(tets[:, j])
    a, b = np.concatenate(a), np.concatenate(b)
    g = sp.csr_matrix((np.ones(len(a), dtype=np.int8), (a, b)), shape=(n_nodes, n_nodes))
    g.sum_duplicates()
    return g


def bandwidth(tets, n_nodes):
    g = node_graph(tets, n_nodes).tocoo()
    return int(np.abs(g.row - g.col).max()) if g.nnz else 0


def rcm_permutation(tets, n_nodes):
    """perm with new node k = old node perm[k] (reverse Cuthill-McKee order)."""
    return np.asarray(reverse_cuthill_mckee(node_graph(tets, n_nodes), symmetric_mode=True), dtype=np.int64)


def morton_permutation(xyz, bits=10):
    """perm with new node k = old node perm[k], in the order of the Morton
    codes of the coordinates quantised to 2^bits cells per axis over the
    mesh's bounding box (bits of x, y, z interleaved, x most significant;
    ties keep the input order)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)
    q = np.minimum((xyz - lo) / span * (1 << bits), (1 << bits) - 1).astype(np.int64)
    code = np.zeros(len(xyz), dtype=np.int64)
    for b in range(bits):
        for axis in range(3):
            code |= ((q[:, axis] >> b) & 1) << (3 * b + 2 - axis)
    return np.argsort(code, kind="stable").astype(np.int64)


def renumber(xyz, tets, perm):
    """The mesh with node k = old node perm[k]: (xyz[perm], tets in new numbers)."""
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    return np.ascontiguousarray(np.asarray(xyz)[perm]), inv[np.asarray(tets)].astype(np.int32)
