"""Whittle-Matern prior by a Fourier spectral method on a box, and RTO in its
latent space (oracle, FP64).  Test infrastructure only: imported by tests/,
never by the library.

Section 4.1.2 (eq. matern-cov-op): C = sigma^2 Z^{-1} (I / l^2 - Laplacian)^{-(s + d/2)}.
Section 6.4: the field is computed spectrally on the cube [-a, a]^3 (a = 2.5,
128^3 points) and carried to the finite element nodes; RTO runs in the latent
Gaussian space of that representation.

Readings (the paper gives the construction in words only):
  * grid x_j = -a + j h, h = 2a / n_g, j = 0..n_g-1, periodic (the box holds
    the computational domain with room to spare, so the wrap-around is outside it);
  * p = P T z with z ~ N(0, I) on the grid, T = F^{-1} diag(sqrt(S)) F (F the
    unitary DFT), S(k) = (1/l^2 + |2 pi k|^2)^{-(s + d/2)} at the DFT
    frequencies k, scaled so that the discrete marginal variance (1/n_g^3) sum S
    is sigma^2 (the normalisation Z);  the covariance of T z is then
    F^{-1} diag(S) F, whose continuum limit for s = 3/2, d = 3 is the Matern
    function sigma^2 (1 + r/l) e^{-r/l};
    (the SPDE written in Section 6.4 applies the cubed operator to p0, which
    would square that covariance; the covariance operator of eq. matern-cov-op
    is followed);
  * P is trilinear interpolation from the grid to the nodes (the paper carries
    the grid field to the finite element space without naming the operator;
    nodal interpolation is the plain reading for a P1 space);
  * latent RTO: min || (G P T z - y_obs) / sigma_n - eta ||^2 + || z - xi ||^2,
    the extended system A = [G P T / sigma_n ; I], b = (y_obs / sigma_n + eta, xi).
"""
from __future__ import annotations

import numpy as np

from . import rto, wave


def grid_axis(n_g, a):
    """The n_g periodic grid coordinates -a + j h, h = 2a / n_g."""
    return -a + (2.0 * a / n_g) * np.arange(n_g)


def spectral_filter(n_g, a, ell, s, sigma, d=3):
    """sqrt(S) on the n_g^3 DFT frequencies, S normalised to marginal variance sigma^2."""
    h = 2.0 * a / n_g
    k = np.fft.fftfreq(n_g, d=h)
    K2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    S = (1.0 / ell ** 2 + 4.0 * np.pi ** 2 * K2) ** (-(s + d / 2.0))
    S *= sigma ** 2 / S.mean()
    return np.sqrt(S)


def apply_T(z, filt):
    """T z = F^{-1} diag(filt) F z over the first three axes (unitary DFTs); a
    real even filter makes T symmetric, so T^T = T."""
    zf = np.fft.fftn(z, axes=(0, 1, 2), norm="ortho")
    f = filt if np.ndim(z) == 3 else filt[..., None]
    return np.real(np.fft.ifftn(f * zf, axes=(0, 1, 2), norm="ortho"))


def grid_covariance(filt):
    """Covariance of T z between grid point 0 and every grid point: the field
    (1/n_g^3) sum_k S(k) e^{2 pi i k x} (inverse DFT of S; at x = 0 the marginal
    variance)."""
    return np.real(np.fft.ifftn(filt ** 2))


def matern_closed_form(r, ell, sigma):
    """Matern covariance for smoothness 3/2 in 3D: sigma^2 (1 + r/l) e^{-r/l}."""
    r = np.asarray(r, dtype=np.float64)
    return sigma ** 2 * (1.0 + r / ell) * np.exp(-r / ell)


def trilinear(n_g, a, xyz):
    """Flat grid indices (N, 8) and trilinear weights (N, 8) of the nodes xyz,
    which must lie in the box [-a, a) on every axis; the grid is periodic, so a
    node above the last grid point a - h interpolates towards the first."""
    h = 2.0 * a / n_g
    u = (np.asarray(xyz, dtype=np.float64) + a) / h
    i0 = np.floor(u).astype(np.int64)
    if np.any(i0 < 0) or np.any(i0 > n_g - 1):
        raise ValueError("node outside the interpolation box")
    f = u - i0
    idx = np.empty((len(u), 8), dtype=np.int64)
    w = np.empty((len(u), 8))
    c = 0
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                ii = (i0 + np.array([dx, dy, dz])) % n_g
                idx[:, c] = (ii[:, 0] * n_g + ii[:, 1]) * n_g + ii[:, 2]
                w[:, c] = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                           * (f[:, 2] if dz else 1 - f[:, 2]))
                c += 1
    return idx, w


def interp(zgrid, idx, w):
    """P z: gather from the grid (flattened) to the nodes."""
    zf = zgrid.reshape(-1, *zgrid.shape[3:])
    if zf.ndim == 1:
        return np.sum(w * zf[idx], axis=1)
    return np.einsum("nc,nck->nk", w, zf[idx])


def interp_T(vals, idx, w, n_g):
    """P^T v: scatter from the nodes to the grid (the transpose of interp)."""
    out = np.zeros((n_g ** 3,) + np.shape(vals)[1:])
    for c in range(idx.shape[1]):
        np.add.at(out, idx[:, c], (w[:, c] if np.ndim(vals) == 1 else w[:, c:c + 1]) * vals)
    return out.reshape((n_g, n_g, n_g) + np.shape(vals)[1:])


def latent_operator(ops, dt, n_steps, sigma_n, filt, idx, w):
    """Actions of A = [G P T / sigma_n ; I] and A^T on latent fields z [n_g]^3(, K)."""
    n_g = filt.shape[0]

    def apply_A(z):
        p = interp(apply_T(z, filt), idx, w)
        return wave.forward(ops, p, dt, n_steps) / sigma_n, np.array(z, dtype=np.float64, copy=True)

    def apply_AT(r):
        r_d, r_p = r
        g = wave.adjoint(ops, r_d, dt) / sigma_n
        return apply_T(interp_T(g, idx, w, n_g), filt) + r_p

    return apply_A, apply_AT


def latent_rto_samples(ops, dt, n_steps, y_obs, sigma_n, eta, xi, filt, idx, w, n_iter, solver="lsqr"):
    """RTO in the latent space: K samples z (latent, [n_g]^3 x K) and the nodal
    samples p = P T z (N x K); eta (N_T, N_obs, K), xi ([n_g]^3, K)."""
    A, AT = latent_operator(ops, dt, n_steps, sigma_n, filt, idx, w)
    b = (np.asarray(y_obs)[..., None] / sigma_n + eta, np.asarray(xi, dtype=np.float64))
    f = rto.lsqr if solver == "lsqr" else rto.cgls
    z, hist = f(A, AT, b, n_iter, np.shape(xi), True)
    return z, interp(apply_T(z, filt), idx, w), hist
