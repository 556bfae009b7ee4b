"""Forward map G and its exact transpose G^T (oracle, FP64).

Forward (Section 3, eq. fully-discrete with M replaced by M_L): per step
    p^{n+1/2} = p^n + dt/2 v^n
    M_L v^{n+1} = M_L v^n - dt K p^{n+1/2} - dt B v^n
    p^{n+1} = p^{n+1/2} + dt/2 v^{n+1}
from z^0 = (p0, 0); observations y^n = Pi p^n for n = 1..N_T (Section 2: t_j =
j dt, j = 1..N_T, no sample at t = 0).  G stacks Pi A^n (eq. discrete-wave-matrix).

Transpose (Section 5.1): zhat^{N_T} = Pi^T yhat^{N_T}, then
zhat^n = Pi^T yhat^n + A^T zhat^{n+1} (eq. backward-recursion), and
G^T yhat = J^T A^T zhat^1 with J p = (p, 0).  One application of A^T is the five
substeps of eq. adjoint-verlet.  Pi^T injects into the pressure block.

All functions accept p0 of shape (N,) or (N, K) (K independent columns) and
observation arrays of shape (N_T, N_obs) or (N_T, N_obs, K).
"""
from __future__ import annotations

import numpy as np


def forward(ops, p0, dt, n_steps):
    """Y = G p0 as an (N_T, N_obs[, K]) array."""
    K, B, ML, Pi = ops["K"], ops["B"], ops["ML"], ops["Pi"]
    p = np.array(p0, dtype=np.float64, copy=True)
    v = np.zeros_like(p)
    mlc = ML if p.ndim == 1 else ML[:, None]
    Y = np.empty((n_steps, Pi.shape[0]) + p.shape[1:])
    for n in range(n_steps):
        p_half = p + 0.5 * dt * v
        v = (mlc * v - dt * (K @ p_half) - dt * (B @ v)) / mlc
        p = p_half + 0.5 * dt * v
        Y[n] = Pi @ p
    return Y


def transpose_step(ops, p_hat, v_hat, dt):
    """One application of A^T to (p_hat, v_hat), eq. adjoint-verlet."""
    K, B, ML = ops["K"], ops["B"], ops["ML"]
    mlc = ML if p_hat.ndim == 1 else ML[:, None]
    p_half = p_hat
    v_half = v_hat + 0.5 * dt * p_hat
    q_half = v_half / mlc
    p_new = p_half - dt * (K.T @ q_half)
    v_new = mlc * q_half - dt * (B.T @ q_half) + 0.5 * dt * p_new
    return p_new, v_new


def adjoint(ops, Yhat, dt):
    """G^T yhat for yhat of shape (N_T, N_obs[, K]); returns the p-block."""
    Pi = ops["Pi"]
    Yhat = np.asarray(Yhat, dtype=np.float64)
    n_steps = Yhat.shape[0]
    p_hat = Pi.T @ Yhat[n_steps - 1]
    v_hat = np.zeros_like(p_hat)
    for n in range(n_steps - 2, -1, -1):
        p_hat, v_hat = transpose_step(ops, p_hat, v_hat, dt)
        p_hat = p_hat + Pi.T @ Yhat[n]
    p_hat, v_hat = transpose_step(ops, p_hat, v_hat, dt)
    return p_hat


def propagator_dense(ops, dt):
    """The one-step propagator A_dt as the dense block matrix of eq. matrix-stromer."""
    K = ops["K"].toarray()
    B = ops["B"].toarray()
    Minv = np.diag(1.0 / ops["ML"])
    N = K.shape[0]
    I = np.eye(N)
    A11 = I - 0.5 * dt ** 2 * Minv @ K
    A12 = dt * I - 0.5 * dt ** 2 * Minv @ B - 0.25 * dt ** 3 * Minv @ K
    A21 = -dt * Minv @ K
    A22 = I - dt * Minv @ B - 0.5 * dt ** 2 * Minv @ K
    return np.block([[A11, A12], [A21, A22]])


def forward_matrix_dense(ops, dt, n_steps):
    """Dense G (N_T*N_obs x N) assembled by columns G e_i (Section 6.1)."""
    N = ops["K"].shape[0]
    Y = forward(ops, np.eye(N), dt, n_steps)      # column i of the identity is e_i
    return Y.reshape(n_steps * Y.shape[1], N)
