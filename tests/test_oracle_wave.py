"""Pins of the oracle's forward map, transpose and stability (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic as S
from oracle import fem, wave


def build(n, n_obs=20, seed=5, faces=S.ALL_FACES):
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, faces, seed)
    return xyz, tets, fem.build(xyz, tets, det, n)


def test_forward_matches_printed_propagator():
    """The three substeps equal powers of the block matrix of eq. matrix-stromer."""
    n = 3
    xyz, tets, ops = build(n)
    dt = 0.3 / n
    N = len(xyz)
    p0 = np.random.default_rng(0).standard_normal(N)
    Y = wave.forward(ops, p0, dt, 25)
    A = wave.propagator_dense(ops, dt)
    z = np.concatenate([p0, np.zeros(N)])
    for t in range(25):
        z = A @ z
        assert np.abs(ops["Pi"] @ z[:N] - Y[t]).max() < 1e-13 * max(1, np.abs(Y).max())


def test_modified_energy_conserved_without_absorption():
    """With B = 0 the drift-kick-drift scheme conserves
    E = 1/2 v^T M_L v - dt^2/8 v^T K v + 1/2 p^T K p exactly (up to rounding)."""
    n = 5
    xyz, tets, ops = build(n)
    N = len(xyz)
    ops = dict(ops)
    ops["B"] = sp.csr_matrix((N, N))
    dt = 0.3 / n
    rng = np.random.default_rng(1)
    p, v = rng.standard_normal(N), rng.standard_normal(N)
    K, ML = ops["K"], ops["ML"]
    energy = lambda p, v: 0.5 * v @ (ML * v) - dt ** 2 / 8 * v @ (K @ v) + 0.5 * p @ (K @ p)
    E0 = energy(p, v)
    for _ in range(300):
        ph = p + 0.5 * dt * v
        v = (ML * v - dt * (K @ ph) - dt * (ops["B"] @ v)) / ML
        p = ph + 0.5 * dt * v
    assert abs(energy(p, v) - E0) / abs(E0) < 1e-13


def test_plane_wave_dispersion_in_the_interior():
    """Away from the boundary the scheme is leapfrog on the 7-point Laplacian, so a
    standing wave u = cos(k.x) started at rest is p^m = cos(m w dt) u with
    cos(w dt) = 1 - dt^2/2 * sum_a 4/h^2 sin^2(k_a h/2) (textbook dispersion relation),
    exactly at nodes the boundary cannot reach in m steps (one node per step)."""
    n = 16
    h = 1.0 / n
    dt = 0.3 * h
    xyz, tets = S.cube_mesh(n)
    ops = fem.assemble(xyz, tets)
    kvec = np.array([2.0, 3.0, 1.0]) * np.pi
    u = np.cos(xyz @ kvec)
    lam = sum(4 / h ** 2 * np.sin(ka * h / 2) ** 2 for ka in kvec)
    wdt = np.arccos(1 - 0.5 * dt ** 2 * lam)
    p, v = u.copy(), np.zeros_like(u)
    m = 5
    for _ in range(m):
        ph = p + 0.5 * dt * v
        v = (ops["ML"] * v - dt * (ops["K"] @ ph) - dt * (ops["B"] @ v)) / ops["ML"]
        p = ph + 0.5 * dt * v
    ijk = np.rint(xyz * n).astype(int)
    deep = np.all((ijk > m) & (ijk < n - m), axis=1)
    assert deep.sum() > 50
    assert np.abs(p[deep] - np.cos(m * wdt) * u[deep]).max() < 1e-12


@pytest.mark.parametrize("n,K", [(3, None), (4, 3)])
def test_dot_product_transpose(n, K):
    """<G p, yhat> = <p, G^T yhat> to machine precision (Section 6.1 adjoint test)."""
    xyz, tets, ops = build(n, n_obs=12)
    dt = 0.3 / n
    rng = np.random.default_rng(2)
    shape = (len(xyz),) if K is None else (len(xyz), K)
    p = rng.standard_normal(shape)
    yhat = rng.standard_normal((40, 12) + shape[1:])
    lhs = np.sum(wave.forward(ops, p, dt, 40) * yhat, axis=(0, 1))
    rhs = np.sum(p * wave.adjoint(ops, yhat, dt), axis=0)
    assert np.all(np.abs(lhs - rhs) <= 1e-13 * np.abs(lhs))


def test_adjoint_equals_dense_transpose():
    n = 2
    xyz, tets, ops = build(n, n_obs=6)
    dt = 0.3 / n
    G = wave.forward_matrix_dense(ops, dt, 15)
    yhat = np.random.default_rng(3).standard_normal((15, 6))
    assert np.abs(wave.adjoint(ops, yhat, dt) - G.T @ yhat.ravel()).max() < 1e-13


@pytest.mark.parametrize("n", [4, 6])
def test_stability_threshold_of_the_explicit_absorbing_term(n):
    """Spectral radius of A_dt: 1 at dt = 0.3 h, > 1 at 0.4 h (the corner nodes)."""
    xyz, tets = S.cube_mesh(n)
    ops = fem.assemble(xyz, tets)
    h = 1.0 / n
    rho = lambda f: np.abs(np.linalg.eigvals(wave.propagator_dense(ops, f * h))).max()
    assert rho(0.3) < 1 + 1e-9
    assert rho(0.34) < 1 + 1e-9
    assert rho(0.35) > 1.01
    assert rho(0.4) > 1.4
    # without the absorbing term every eigenvalue lies on the unit circle at 0.4 h
    ops0 = dict(ops)
    ops0["B"] = 0 * ops["B"]
    assert abs(np.abs(np.linalg.eigvals(wave.propagator_dense(ops0, 0.4 * h))).max() - 1) < 1e-9
