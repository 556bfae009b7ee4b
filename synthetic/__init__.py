"""Seeded synthetic inputs for the photoacoustic RTO workloads.

This module only *makes inputs*: tetrahedral cube meshes, detector points on the
cube faces, initial-pressure phantoms and the standard-normal draws that the RTO
sampler consumes.  It holds none of the method's arithmetic (no assembly, no
time stepping, no adjoint, no least squares), so that both the CPU oracle and
the CUDA library can be fed from it without sharing any of the computation.

The paper measures on a sphere of radius 2 with ~2e5 unknowns (Section 6.4);
its meshes and phantoms are not published, so the workloads here are seeded
stand-ins with the same sizes: a unit cube split into Kuhn tetrahedra, detectors
at random points on five or six faces, Gaussian blobs plus a vessel tree.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

# ----------------------------------------------------------------------------
# Mesh
# ----------------------------------------------------------------------------

# The six axis permutations in lexicographic order; each gives one tetrahedron
# of a cube cell as the monotone lattice path v0 -> +e_a -> +e_a+e_b -> v0+(1,1,1).
KUHN_PERMUTATIONS = tuple(itertools.permutations((0, 1, 2)))


def node_index(i, j, k, n):
    """Node number of lattice point (i, j, k) on an n^3-cell cube (k fastest)."""
    return (i * (n + 1) + j) * (n + 1) + k


def cube_mesh(n: int):
    """Unit cube [0,1]^3, n^3 cells, each split into 6 Kuhn tetrahedra.

    Returns ``(xyz, tets)``: xyz is (N, 3) float64 with N = (n+1)^3 and node
    (i, j, k) at (i/n, j/n, k/n); tets is (6 n^3, 4) int32, cells in (i, j, k)
    order with k fastest, the 6 tets of a cell in the order of
    ``KUHN_PERMUTATIONS``, vertices in lattice-path order.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    g = np.arange(n + 1, dtype=np.float64) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for t, perm in enumerate(KUHN_PERMUTATIONS):
        off = np.zeros(3, dtype=np.int64)
        tets[:, t, 0] = node_index(ci, cj, ck, n)
        for s, axis in enumerate(perm):
            off[axis] += 1
            tets[:, t, s + 1] = node_index(ci + off[0], cj + off[1], ck + off[2], n)
    return xyz, tets.reshape(-1, 4).astype(np.int32)


def jittered_cube_mesh(n: int, amp: float, seed: int):
    """cube_mesh(n) with every interior node moved by amp * h * U[-1, 1] per
    coordinate (h = 1 / n; seeded), boundary nodes left on the lattice so the
    faces stay planar.  The connectivity is the Kuhn one, but no stiffness entry
    cancels any more: an interior row couples its node to all 14 graph
    neighbours, as on the paper's unstructured meshes (Section 6.4).  amp <= 0.15
    keeps every tetrahedron's orientation (checked).  Returns (xyz, tets)."""
    if not 0.0 <= amp <= 0.15:
        raise ValueError("amp must be in [0, 0.15]")
    xyz, tets = cube_mesh(n)
    rng = np.random.default_rng(seed)
    d = rng.uniform(-1.0, 1.0, size=xyz.shape) * (amp / n)
    interior = np.all((xyz > 0.5 / n) & (xyz < 1.0 - 0.5 / n), axis=1)
    def orient(p):
        X = p[tets]
        return np.einsum("ei,ei->e", np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), X[:, 3] - X[:, 0])

    before = orient(xyz)
    xyz = xyz + d * interior[:, None]
    if not np.all(orient(xyz) * before > 0.0):
        raise ValueError("jitter inverted a tetrahedron")
    return xyz, tets


def sphere_mesh(n: int, radius: float):
    """A ball of the given radius carved from the Kuhn mesh of [-radius, radius]^3
    with n cells per side: the tetrahedra whose centroid lies inside the ball,
    the nodes they use renumbered in their lexicographic order.  A stand-in for
    the paper's unstructured sphere mesh (Section 6.4), whose mesher and mesh
    are not available: a stair-cased boundary, interior nodes of graph degree
    up to 14.  Returns (xyz, tets) as cube_mesh does."""
    xyz, tets = cube_mesh(n)
    xyz = (2.0 * xyz - 1.0) * radius
    cent = xyz[tets].mean(axis=1)
    keep = np.einsum("ij,ij->i", cent, cent) < radius * radius
    tets = tets[keep]
    used = np.unique(tets)
    new = -np.ones(len(xyz), dtype=np.int64)
    new[used] = np.arange(len(used))
    return xyz[used], new[tets].astype(np.int32)


def octant_node_sensors(xyz, n_obs: int, r_phys: float, h: float, seed: int):
    """Node-coincident detectors on the physical sphere of radius r_phys, first
    octant (Section 6.4): n_obs seeded picks among the nodes with x, y, z >= 0
    whose radius is within h / 2 of r_phys.  Returns their coordinates (n_obs, 3)."""
    r = np.linalg.norm(xyz, axis=1)
    cand = np.nonzero((np.abs(r - r_phys) <= 0.5 * h) & np.all(xyz >= 0.0, axis=1))[0]
    if len(cand) < n_obs:
        raise ValueError(f"only {len(cand)} candidate nodes for {n_obs} detectors")
    pick = np.random.default_rng(seed).choice(cand, size=n_obs, replace=False)
    return xyz[np.sort(pick)]


def octant_sphere_points(n_obs: int, r_phys: float, seed: int):
    """Detectors on the physical sphere of radius r_phys, first octant (Section
    6.4), uniform on that spherical triangle (seeded): generally inside a
    tetrahedron of the mesh, not at a node."""
    rng = np.random.default_rng(seed)
    v = np.abs(rng.standard_normal((n_obs, 3)))
    return r_phys * v / np.linalg.norm(v, axis=1, keepdims=True)


# ----------------------------------------------------------------------------
# Detectors
# ----------------------------------------------------------------------------

# Face f: axis f // 2 fixed at value f % 2 (0: x=0, 1: x=1, 2: y=0, ... 5: z=1).
ALL_FACES = (0, 1, 2, 3, 4, 5)
LIMITED_VIEW_FACES = (0, 1, 2, 3, 4)  # z = 1 left open


def detector_points(n_obs: int, faces, seed: int):
    """``n_obs`` points drawn uniformly on the listed cube faces.

    The face is drawn uniformly from ``faces``; the two in-plane coordinates
    (in increasing axis order) are U[0,1).  Returns (n_obs, 3) float64.
    """
    rng = np.random.default_rng(seed)
    faces = np.asarray(faces)
    f = faces[rng.integers(0, len(faces), size=n_obs)]
    uv = rng.random((n_obs, 2))
    pts = np.empty((n_obs, 3))
    for d in range(n_obs):
        axis, side = divmod(int(f[d]), 2)
        others = [a for a in range(3) if a != axis]
        pts[d, axis] = float(side)
        pts[d, others[0]] = uv[d, 0]
        pts[d, others[1]] = uv[d, 1]
    return pts


# ----------------------------------------------------------------------------
# Phantoms
# ----------------------------------------------------------------------------

def gaussian_blobs(xyz, n_blobs: int, seed: int, sigma=(0.1, 0.1), amp=(0.5, 1.0),
                   centre=(0.2, 0.8)):
    """Sum of isotropic Gaussian blobs evaluated at the nodes."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(centre[0], centre[1], size=(n_blobs, 3))
    s = rng.uniform(sigma[0], sigma[1], size=n_blobs)
    a = rng.uniform(amp[0], amp[1], size=n_blobs)
    p = np.zeros(len(xyz))
    for b in range(n_blobs):
        r2 = np.sum((xyz - c[b]) ** 2, axis=1)
        p += a[b] * np.exp(-r2 / (2.0 * s[b] ** 2))
    return p


def vessel_tree(xyz, seed: int, depth: int = 4, h: float = 1.0 / 32):
    """A seeded binary tree of tubes, max-combined, with a Gaussian profile.

    Root at (0.5, 0.5, 0.15) heading +z; segment length 0.25 * 0.75^level,
    branches turned by +-35 degrees about a random axis, tube radius
    0.015 * 0.8^level widened to at least the mesh width h (the smoothing).
    """
    rng = np.random.default_rng(seed)
    segs = []

    def grow(p, d, level):
        if level > depth:
            return
        length = 0.25 * 0.75 ** level
        q = p + length * d
        segs.append((p.copy(), q.copy(), 0.015 * 0.8 ** level))
        for sgn in (-1.0, 1.0):
            axis = rng.normal(size=3)
            axis -= axis.dot(d) * d
            axis /= np.linalg.norm(axis)
            ang = sgn * math.radians(35.0)
            nd = d * math.cos(ang) + np.cross(axis, d) * math.sin(ang)
            grow(q, nd / np.linalg.norm(nd), level + 1)

    grow(np.array([0.5, 0.5, 0.15]), np.array([0.0, 0.0, 1.0]), 0)
    val = np.zeros(len(xyz))
    for p, q, r in segs:
        d = q - p
        t = np.clip(((xyz - p) @ d) / d.dot(d), 0.0, 1.0)
        dist2 = np.sum((xyz - (p + t[:, None] * d)) ** 2, axis=1)
        w = max(r, h)
        val = np.maximum(val, 0.8 * np.exp(-dist2 / (2.0 * w * w)))
    return val


def phantom(xyz, kind: str, seed: int, n: int):
    """Initial pressure of the workloads: 'blobs3' or 'blobs20+vessels'."""
    if kind == "blobs3":
        return gaussian_blobs(xyz, 3, seed, sigma=(0.1, 0.1))
    if kind == "blobs20+vessels":
        p = gaussian_blobs(xyz, 20, seed, sigma=(0.03, 0.08))
        return np.maximum(p, vessel_tree(xyz, seed + 1, h=1.0 / n))
    raise ValueError(kind)


def smoothed_speed_field(n: int, seed: int, amplitude: float = 0.1):
    """Per-tet sound speed c = 1 + amplitude * z, z a box-filtered N(0,1) cell field.

    z is drawn per cell, box-filtered 3x3x3 three times (edge-replicated),
    renormalised to zero mean and unit std; the 6 tets of a cell share it.
    Returns c^2 per tet, float64 of length 6 n^3 (cell order of ``cube_mesh``).
    """
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n, n, n))
    for _ in range(3):
        zp = np.pad(z, 1, mode="edge")
        acc = np.zeros_like(z)
        for a in range(3):
            for b in range(3):
                for c in range(3):
                    acc += zp[a:a + n, b:b + n, c:c + n]
        z = acc / 27.0
    z = (z - z.mean()) / z.std()
    c = 1.0 + amplitude * z.ravel()
    return np.repeat(c * c, 6)


# ----------------------------------------------------------------------------
# Random draws consumed by the sampler
# ----------------------------------------------------------------------------

def standard_normal(shape, seed: int, dtype=np.float64):
    """Seeded i.i.d. N(0,1) array (PCG64)."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def device_standard_normal(shape, seed: int, device):
    """Seeded i.i.d. N(0,1) float32 tensor drawn on a torch device (for inputs
    too large to draw on the host); the tests read back the columns they check."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    return torch.randn(shape, generator=gen, device=device, dtype=torch.float32)


# ----------------------------------------------------------------------------
# Workload definitions
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int                 # cells per cube edge
    n_steps: int           # N_T
    dt_factor: float       # dt = dt_factor * h / c_max
    n_obs: int
    faces: tuple
    phantom: str
    noise: float           # relative noise level d_noise
    K: int                 # stacked RTO samples
    n_iter: int            # CGLS iterations
    precision: str         # "f64" or "f32"
    seed: int

    @property
    def h(self):
        return 1.0 / self.n

    @property
    def n_nodes(self):
        return (self.n + 1) ** 3

    @property
    def dt(self):
        return self.dt_factor * self.h


# Time step 0.3 h everywhere: 0.4 h is unstable with the explicit absorbing
# term on a cube (the corner nodes), see the stability tests.
SMALL_F64 = Workload("cube8_fp64", 8, 200, 0.3, 32, ALL_FACES, "blobs3", 0.01, 16, 50, "f64", 1001)
PLAIN_F32 = Workload("cube32_fp32", 32, 600, 0.3, 256, LIMITED_VIEW_FACES, "blobs20+vessels",
                     0.01, 1, 100, "f32", 1002)
BATCHED = Workload("cube58_batched", 58, 1000, 0.3, 1024, LIMITED_VIEW_FACES, "blobs20+vessels",
                   0.01, 64, 100, "f32", 1003)
DIFFERENTIATION = Workload("cube32_grad", 32, 1000, 0.3, 256, LIMITED_VIEW_FACES, "blobs20+vessels",
                           0.01, 1, 0, "f32", 1004)
UNEVEN = tuple(
    Workload(f"cube{n}_uneven", n, int(round(1000 * n / 58)), 0.3, int(round(1024 * (n / 58) ** 2)),
             LIMITED_VIEW_FACES, "blobs20+vessels", d, K, 50, "f32", 1005 + 10 * i)
    for i, (n, K, d) in enumerate(zip((16, 24, 32, 40, 48, 58), (256, 128, 64, 32, 16, 8),
                                      (0.01, 0.02, 0.03, 0.04, 0.01, 0.02)))
)


def make_problem(w: Workload):
    """Mesh, detector points and true initial pressure for a workload."""
    xyz, tets = cube_mesh(w.n)
    det = detector_points(w.n_obs, w.faces, w.seed)
    p0 = phantom(xyz, w.phantom, w.seed + 100, w.n)
    return xyz, tets, det, p0
