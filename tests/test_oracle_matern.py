"""Pins of the Whittle-Matern oracle (oracle/matern.py): the closed-form Matern
covariance, the square-root filter, trilinear interpolation and its transpose,
and latent-space RTO against a dense solve and SciPy's LSQR (CPU only)."""
import numpy as np
import pytest

import synthetic as S
from oracle import fem, matern as M, rto, wave


def test_grid_covariance_is_the_matern_function():
    """For s = 3/2 in 3D the covariance of (1/l^2 - Laplacian)^{-3} is
    sigma^2 (1 + r/l) e^{-r/l}; the spectral grid reproduces it, better on finer grids."""
    errs = []
    for n_g, ell in ((64, 0.3), (32, 0.5), (64, 0.5), (128, 0.5)):
        filt = M.spectral_filter(n_g, 2.5, ell, 1.5, 3.0)
        c = M.grid_covariance(filt)
        h = 5.0 / n_g
        j = np.arange(12)
        assert abs(c[0, 0, 0] - 9.0) < 1e-12                           # marginal variance sigma^2
        for lag in (c[j, 0, 0], c[0, j, 0], c[0, 0, j]):
            err = np.abs(lag - M.matern_closed_form(j * h, ell, 3.0)).max() / 9.0
            errs.append(err)
        assert abs(c[2, 1, 0] - M.matern_closed_form(np.sqrt(5) * h, ell, 3.0)) / 9.0 < 2e-2
    assert errs[0] < 1e-3                                             # l = 0.3 on 64^3
    assert errs[3] > errs[6] > errs[9]                                # l = 0.5: 32^3 -> 64^3 -> 128^3


def test_T_is_the_square_root_of_the_covariance_and_symmetric():
    filt = M.spectral_filter(16, 2.5, 0.4, 1.5, 2.0)
    delta = np.zeros((16, 16, 16))
    delta[0, 0, 0] = 1.0
    assert np.abs(M.apply_T(M.apply_T(delta, filt), filt) - M.grid_covariance(filt)).max() < 1e-12
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal((16, 16, 16)), rng.standard_normal((16, 16, 16))
    assert abs(np.sum(M.apply_T(a, filt) * b) - np.sum(a * M.apply_T(b, filt))) < 1e-10 * np.sqrt(np.sum(a * a))
    K = rng.standard_normal((16, 16, 16, 3))
    assert np.abs(M.apply_T(K, filt)[..., 1] - M.apply_T(K[..., 1], filt)).max() < 1e-13


def test_trilinear_interpolation_and_its_transpose():
    xyz, _ = S.sphere_mesh(6, 2.0)
    n_g, a = 16, 2.5
    idx, w = M.trilinear(n_g, a, xyz)
    assert np.abs(w.sum(axis=1) - 1.0).max() < 1e-14 and np.all(w >= -1e-15)
    x = M.grid_axis(n_g, a)
    G = np.meshgrid(x, x, x, indexing="ij")
    f = 0.3 * G[0] - 1.1 * G[1] + 0.7 * G[2] + 0.2                   # affine: reproduced exactly
    assert np.abs(M.interp(f, idx, w) - (xyz @ np.array([0.3, -1.1, 0.7]) + 0.2)).max() < 1e-13
    rng = np.random.default_rng(2)
    g, v = rng.standard_normal((n_g, n_g, n_g)), rng.standard_normal(len(xyz))
    assert abs(np.dot(M.interp(g, idx, w), v) - np.sum(g * M.interp_T(v, idx, w, n_g))) < 1e-11
    with pytest.raises(ValueError):
        M.trilinear(n_g, a, np.array([[2.51, 0.0, 0.0]]))
    # above the last grid point the periodic grid wraps: a periodic field is reproduced
    h = 2 * a / n_g
    top = np.array([[a - 0.5 * h, 0.1, -0.3]])
    ti, tw = M.trilinear(n_g, a, top)
    cosf = np.cos(np.pi * G[0] / a)                                   # period 2a
    assert abs(M.interp(cosf, ti, tw)[0] - 0.5 * (np.cos(np.pi * (a - h) / a) + np.cos(-np.pi))) < 1e-14


def _latent_problem(n_g=6, K=2):
    xyz, tets = S.sphere_mesh(4, 2.0)
    det = S.octant_node_sensors(xyz, 6, 1.0, 1.0, 3)
    ops = fem.build_node_sensors(xyz, tets, det)
    dt, nt = 0.2, 20
    filt = M.spectral_filter(n_g, 2.5, 0.6, 1.5, 1.0)
    idx, w = M.trilinear(n_g, 2.5, xyz)
    p0 = S.gaussian_blobs(xyz, 2, 4, sigma=(0.4, 0.6), centre=(-0.5, 0.5))
    Y = wave.forward(ops, p0, dt, nt)
    y_obs, sig = rto.add_noise(Y, S.standard_normal(Y.shape, 5), 0.05, dt)
    eta = S.standard_normal((nt, 6, K), 6)
    xi = S.standard_normal((n_g, n_g, n_g, K), 7)
    return ops, dt, nt, y_obs, sig, eta, xi, filt, idx, w


def _dense_latent(ops, dt, nt, sig, filt, idx, w):
    n_g = filt.shape[0]
    G = wave.forward_matrix_dense(ops, dt, nt)
    Ng = n_g ** 3
    E = np.eye(Ng).reshape(n_g, n_g, n_g, Ng)
    PT = M.interp(M.apply_T(E, filt), idx, w)                          # (N, Ng)
    return np.vstack([G @ PT / sig, np.eye(Ng)]), PT


def test_latent_rto_converges_to_the_dense_least_squares_solution():
    ops, dt, nt, y, sig, eta, xi, filt, idx, w = _latent_problem()
    A, PT = _dense_latent(ops, dt, nt, sig, filt, idx, w)
    z, p, hist = M.latent_rto_samples(ops, dt, nt, y, sig, eta, xi, filt, idx, w, 300)
    for k in range(2):
        b = np.concatenate([(y / sig + eta[..., k]).ravel(), xi[..., k].ravel()])
        ref = np.linalg.lstsq(A, b, rcond=None)[0]
        assert np.linalg.norm(z[..., k].ravel() - ref) <= 1e-8 * np.linalg.norm(ref)
        assert np.linalg.norm(p[:, k] - PT @ ref) <= 1e-8 * np.linalg.norm(PT @ ref)


def test_latent_rto_iterates_equal_scipy_lsqr_and_cgls():
    from scipy.sparse.linalg import lsqr as sp_lsqr
    ops, dt, nt, y, sig, eta, xi, filt, idx, w = _latent_problem(K=1)
    A, _ = _dense_latent(ops, dt, nt, sig, filt, idx, w)
    b = np.concatenate([(y / sig + eta[..., 0]).ravel(), xi[..., 0].ravel()])
    for k in (1, 2, 3):
        z, _, _ = M.latent_rto_samples(ops, dt, nt, y, sig, eta, xi, filt, idx, w, k)
        ref = sp_lsqr(A, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k)[0]
        assert np.linalg.norm(z[..., 0].ravel() - ref) <= 1e-9 * np.linalg.norm(ref)
        zc, _, _ = M.latent_rto_samples(ops, dt, nt, y, sig, eta, xi, filt, idx, w, k, solver="cgls")
        assert np.linalg.norm(zc - z) <= 1e-9 * np.linalg.norm(z)
