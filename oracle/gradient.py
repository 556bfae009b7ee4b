"""Derivatives of a data misfit through the forward map (oracle, FP64).

Misfit L(p0, theta) = 1/2 ||G(theta) p0 - y||^2 with K(theta) = sum_e theta_e K_e^0,
theta_e = c_e^2 (K_e^0 the c = 1 element stiffness of Section 3).

dL/dp0 = G^T (G p0 - y) by the backward recursion of Section 5.1.
dL/dtheta_e: the only place theta enters one Stoermer-Verlet step is the
velocity update M_L v^{n+1} = M_L v^n - dt K p^{n+1/2} - dt B v^n, so with
vhat^{n+1/2} the cotangent of that v^{n+1} (second line of eq. adjoint-verlet)
and qhat = M_L^{-1} vhat^{n+1/2} (third line),
    dL/dtheta_e = -dt sum_n qhat_e^T K_e^0 p_e^{n+1/2},
where _e restricts to the element's four nodes.  The oracle stores the whole
forward trajectory (no checkpointing); ``misfit`` lets the tests check both
derivatives by central finite differences.
"""
from __future__ import annotations

import numpy as np

from . import fem, wave


def element_stiffness_unit(ops):
    """K_e^0 = V grad(lambda_a) . grad(lambda_b) for every element, (E, 4, 4)."""
    return ops["vol"][:, None, None] * np.einsum("eai,ebi->eab", ops["grads"], ops["grads"])


def with_c2(ops, tets, c2_elem):
    """Copy of ``ops`` with K re-assembled for per-element c^2 (B unchanged)."""
    new = dict(ops)
    Ke = np.asarray(c2_elem)[:, None, None] * element_stiffness_unit(ops)
    N = ops["K"].shape[0]
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    import scipy.sparse as sp
    new["K"] = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(N, N))
    new["c2"] = np.asarray(c2_elem, dtype=np.float64)
    return new


def misfit(ops, p0, y, dt):
    """L = 1/2 ||G p0 - y||^2."""
    r = wave.forward(ops, p0, dt, y.shape[0]) - y
    return 0.5 * float(np.sum(r * r))


def gradients(ops, tets, p0, y, dt):
    """(dL/dp0, dL/dtheta) for L = 1/2 ||G p0 - y||^2 (single sample, p0 of shape (N,))."""
    K, B, ML, Pi = ops["K"], ops["B"], ops["ML"], ops["Pi"]
    n_steps = y.shape[0]
    # forward, keeping p^{n+1/2} of every step
    p = np.array(p0, dtype=np.float64, copy=True)
    v = np.zeros_like(p)
    halves = []
    Y = np.empty_like(y)
    for n in range(n_steps):
        p_half = p + 0.5 * dt * v
        halves.append(p_half)
        v = (ML * v - dt * (K @ p_half) - dt * (B @ v)) / ML
        p = p_half + 0.5 * dt * v
        Y[n] = Pi @ p
    yhat = Y - y
    Ke0 = element_stiffness_unit(ops)
    g_theta = np.zeros(len(tets))

    def reverse_step(p_hat, v_hat, p_half):
        # eq. adjoint-verlet, plus the theta contribution of this step
        v_half = v_hat + 0.5 * dt * p_hat
        q_half = v_half / ML
        qe = q_half[tets]                                  # (E, 4)
        pe = p_half[tets]
        g_theta[:] += -dt * np.einsum("ea,eab,eb->e", qe, Ke0, pe)
        p_new = p_hat - dt * (K.T @ q_half)
        v_new = ML * q_half - dt * (B.T @ q_half) + 0.5 * dt * p_new
        return p_new, v_new

    p_hat = Pi.T @ yhat[n_steps - 1]
    v_hat = np.zeros_like(p_hat)
    for n in range(n_steps - 1, 0, -1):
        p_hat, v_hat = reverse_step(p_hat, v_hat, halves[n])
        p_hat = p_hat + Pi.T @ yhat[n - 1]
    p_hat, v_hat = reverse_step(p_hat, v_hat, halves[0])
    return p_hat, g_theta


__all__ = ["element_stiffness_unit", "with_c2", "misfit", "gradients", "fem"]
