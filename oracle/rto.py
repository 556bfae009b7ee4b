"""Noise model, CGLS, randomize-then-optimize and posterior statistics (oracle, FP64).

Section 2 (eq. noise-model): eta = d ||Y|| / ||eta0|| eta0 with the discrete
L2(0,T; l2) norm ||Y|| = (dt sum_j sum_i Y_ji^2)^{1/2}; sigma = d ||Y|| / ||eta0||
(Section 4.2).

Section 5 (eq. optimization, eq. extended-matrices): with the independent
Gaussian prior C = M_L^{-1} (Section 4.1.1, eq. iid-prior), one RTO sample is
the least-squares solution of G_ext p = b with
    G_ext = [sigma^{-1} G ; M_L^{1/2}],
    b     = [sigma^{-1}(y_obs + sigma eta) ; M_L^{1/2} p_prior],
    p_prior = C^{1/2} xi = M_L^{-1/2} xi,  eta, xi ~ N(0, I).
The least-squares problem is solved by CGLS or by LSQR (Paige & Saunders 1982,
the paper's solver; the paper allows either, eq. normal-equations) started from
x = 0 with a fixed number of iterations (the paper uses fixed iteration limits,
Section 6.1), Algorithm 1.  In exact arithmetic both produce the same iterates
(the minimiser of ||A x - b|| over the k-th Krylov space of A^T A and A^T b).
MAP (eq. MAP) is the same problem with zero perturbations.  The data-space
norm is the plain Euclidean one (the dt of the L2(0,T) norm cancels in sigma).

Statistics: eq. ergodic (mean, and std with 1/(N_sample - 1)).
Dense posterior for small meshes: Appendix A, C_post = (G^T G / sigma^2 + C^{-1})^{-1},
mu_post = C_post G^T y / sigma^2, and the exact sample formula
p = C_post [G^T y / sigma^2 + G^T eta / sigma + L^T L p_prior].
"""
from __future__ import annotations

import numpy as np

from . import wave


def l2_time_norm(Y, dt):
    """Discrete L2(0,T; l2) norm of a space-time array (eq. noise-model)."""
    return np.sqrt(dt * np.sum(np.asarray(Y, dtype=np.float64) ** 2))


def add_noise(Y, eta0, d_noise, dt):
    """Observed data and sigma: y_obs = Y + eta, eta = d ||Y|| / ||eta0|| eta0."""
    sigma = d_noise * l2_time_norm(Y, dt) / l2_time_norm(eta0, dt)
    return Y + sigma * eta0, sigma


def _colsum(a):
    """Sum over all axes but the last one when batched (K columns), else all."""
    return np.sum(a.reshape(-1, a.shape[-1]), axis=0)


def _sq(blocks, batched):
    if batched:
        return sum(_colsum(u * u) for u in blocks)
    return sum(float(np.sum(u * u)) for u in blocks)


def cgls_begin(apply_AT, b, x_shape, batched):
    """CGLS start from x = 0: r = b, s = A^T r, d = s, gamma = ||s||^2."""
    r = tuple(np.array(u, dtype=np.float64, copy=True) for u in b)
    s = apply_AT(r)
    return {"x": np.zeros(x_shape), "r": r, "s": s, "d": s.copy(), "gamma": _sq((s,), batched)}


def cgls_step(apply_A, apply_AT, st, batched):
    """One CGLS iteration (Hestenes-Stiefel CG on the normal equations):
    q = A d; alpha = gamma / ||q||^2; x += alpha d; r -= alpha q;
    s = A^T r; gamma' = ||s||^2; beta = gamma' / gamma; d = s + beta d."""
    q = apply_A(st["d"])
    alpha = st["gamma"] / _sq(q, batched)
    x = st["x"] + alpha * st["d"]
    r = tuple(ri - alpha * qi for ri, qi in zip(st["r"], q))
    s = apply_AT(r)
    gamma = _sq((s,), batched)
    beta = gamma / st["gamma"]
    return {"x": x, "r": r, "s": s, "d": s + beta * st["d"], "gamma": gamma}


def cgls(apply_A, apply_AT, b, n_iter, x_shape, batched, block_hist=False):
    """CGLS for min ||A x - b||_2 from x = 0, exactly n_iter iterations.

    Textbook form (Hestenes-Stiefel CG on the normal equations, as in Hansen,
    Rank-Deficient and Discrete Ill-Posed Problems, 1998).  ``b`` and ``q`` are
    tuples of blocks; with ``batched`` every array carries K independent
    problems in its last axis and the scalars are per column.
    Returns x and the history of ||r||^2 (one entry per iterate); with
    ``block_hist`` the squared norm of each block of r separately, stacked in
    a last axis (the data misfit and prior terms of the Section 6.1 diagnostics).
    """
    def record(r):
        return [_sq((u,), batched) for u in r] if block_hist else _sq(r, batched)

    st = cgls_begin(apply_AT, b, x_shape, batched)
    hist = [record(st["r"])]
    for _ in range(n_iter):
        st = cgls_step(apply_A, apply_AT, st, batched)
        hist.append(record(st["r"]))
    h = np.array(hist)
    return st["x"], (np.moveaxis(h, 1, -1) if block_hist and batched else h)


def _div(a, b):
    """a / b per column, 0 where b == 0 (a Golub-Kahan vector of norm 0 stays 0)."""
    b = np.asarray(b, dtype=np.float64)
    return np.where(b != 0.0, a / np.where(b != 0.0, b, 1.0), 0.0)


def lsqr_begin(apply_AT, b, x_shape, batched):
    """LSQR start (Paige & Saunders 1982, the paper's solver, Section 5.1):
    beta_1 u_1 = b, alpha_1 v_1 = A^T u_1, w_1 = v_1, x_0 = 0,
    phibar_1 = beta_1, rhobar_1 = alpha_1."""
    beta = np.sqrt(_sq(b, batched))
    u = tuple(_div(np.asarray(ui, dtype=np.float64), beta) for ui in b)
    vh = apply_AT(u)
    alpha = np.sqrt(_sq((vh,), batched))
    v = _div(vh, alpha)
    return {"x": np.zeros(x_shape), "u": u, "v": v, "w": v.copy(), "alpha": alpha,
            "phibar": beta, "rhobar": alpha}


def lsqr_step(apply_A, apply_AT, st, batched):
    """One LSQR iteration: Golub-Kahan bidiagonalization
        beta u' = A v - alpha u,   alpha' v' = A^T u' - beta v,
    the plane rotation that eliminates beta from the lower bidiagonal
        rho = (rhobar^2 + beta^2)^{1/2}, c = rhobar / rho, s = beta / rho,
        theta = s alpha', rhobar' = -c alpha', phi = c phibar, phibar' = s phibar,
    and the updates x += (phi / rho) w, w = v' - (theta / rho) w.
    phibar' is the norm of the residual b - A x of the new iterate."""
    Av = apply_A(st["v"])
    uh = tuple(a - st["alpha"] * u for a, u in zip(Av, st["u"]))
    beta = np.sqrt(_sq(uh, batched))
    u = tuple(_div(x, beta) for x in uh)
    vh = apply_AT(u) - beta * st["v"]
    alpha = np.sqrt(_sq((vh,), batched))
    v = _div(vh, alpha)
    rho = np.sqrt(st["rhobar"] ** 2 + beta ** 2)
    c, s = _div(st["rhobar"], rho), _div(beta, rho)
    theta, rhobar = s * alpha, -c * alpha
    phi, phibar = c * st["phibar"], s * st["phibar"]
    x = st["x"] + _div(phi, rho) * st["w"]
    w = v - _div(theta, rho) * st["w"]
    return {"x": x, "u": u, "v": v, "w": w, "alpha": alpha, "phibar": phibar, "rhobar": rhobar}


def lsqr(apply_A, apply_AT, b, n_iter, x_shape, batched):
    """LSQR for min ||A x - b||_2 from x = 0, exactly n_iter iterations (the
    paper's fixed iteration limits, Section 6.1).  Same block / batched
    conventions as cgls.  Returns x and the history of phibar = ||b - A x||
    (one entry per iterate, starting with ||b||)."""
    st = lsqr_begin(apply_AT, b, x_shape, batched)
    hist = [st["phibar"]]
    for _ in range(n_iter):
        st = lsqr_step(apply_A, apply_AT, st, batched)
        hist.append(st["phibar"])
    return st["x"], np.array(hist)


def extended_operator(ops, dt, n_steps, sigma):
    """Actions of G_ext and G_ext^T (eq. lsqr-residual, eq. lsqr-transpose-action)."""
    ML = ops["ML"]

    def sqrt_ml(p):
        return (np.sqrt(ML) if p.ndim == 1 else np.sqrt(ML)[:, None]) * p

    def apply_A(p):
        return (wave.forward(ops, p, dt, n_steps) / sigma, sqrt_ml(p))

    def apply_AT(r):
        r_d, r_p = r
        return wave.adjoint(ops, r_d, dt) / sigma + sqrt_ml(r_p)

    return apply_A, apply_AT


def rto_rhs(ops, y_obs, sigma, eta, xi):
    """Right-hand side b of eq. extended-matrices for given draws eta, xi.

    y_obs (N_T, N_obs); eta (N_T, N_obs[, K]); xi (N[, K]).
    """
    ML = ops["ML"]
    batched = np.ndim(xi) == 2
    mlc = ML[:, None] if batched else ML
    yo = y_obs[..., None] if batched else y_obs
    p_prior = xi / np.sqrt(mlc)                      # C^{1/2} xi with C = M_L^{-1}
    return ((yo + sigma * eta) / sigma, np.sqrt(mlc) * p_prior)


def rto_samples(ops, dt, n_steps, y_obs, sigma, eta, xi, n_iter, block_hist=False):
    """RTO posterior samples (Algorithm 1) for K draws stacked in the last axis.

    Returns samples (N, K) and the CGLS residual history (n_iter+1, K), or with
    ``block_hist`` its data and prior blocks (n_iter+1, K, 2).
    """
    apply_A, apply_AT = extended_operator(ops, dt, n_steps, sigma)
    b = rto_rhs(ops, y_obs, sigma, eta, xi)
    batched = np.ndim(xi) == 2
    return cgls(apply_A, apply_AT, b, n_iter, np.shape(xi), batched, block_hist)


def rto_samples_lsqr(ops, dt, n_steps, y_obs, sigma, eta, xi, n_iter):
    """RTO samples as Algorithm 1 states them, with LSQR.  Returns samples and
    the phibar history (n_iter + 1, K)."""
    apply_A, apply_AT = extended_operator(ops, dt, n_steps, sigma)
    b = rto_rhs(ops, y_obs, sigma, eta, xi)
    return lsqr(apply_A, apply_AT, b, n_iter, np.shape(xi), np.ndim(xi) == 2)


def map_estimate(ops, dt, n_steps, y_obs, sigma, n_iter, solver="lsqr"):
    """MAP estimate (eq. MAP): the extended least-squares problem with zero
    perturbations, b = (y_obs / sigma, 0); returns x and the residual history."""
    apply_A, apply_AT = extended_operator(ops, dt, n_steps, sigma)
    b = (np.asarray(y_obs, dtype=np.float64) / sigma, np.zeros(len(ops["ML"])))
    f = lsqr if solver == "lsqr" else cgls
    return f(apply_A, apply_AT, b, n_iter, (len(ops["ML"]),), False)


def whitened_misfit(ops, dt, n_steps, p, y_obs, sigma):
    """Discrepancy-principle diagnostic (Section 6.1): ||G p - y_obs|| / (sigma
    sqrt(N_T N_obs)), about 1 when the data are fitted to the noise level."""
    r = wave.forward(ops, p, dt, n_steps) - (y_obs if np.ndim(p) == 1 else np.asarray(y_obs)[..., None])
    n = np.prod(np.shape(y_obs))
    if np.ndim(p) == 1:
        return np.sqrt(np.sum(r * r)) / (sigma * np.sqrt(n))
    return np.sqrt(_colsum(r * r)) / (sigma * np.sqrt(n))


def ergodic_mean_std(samples):
    """Pointwise mean and std (1/(N_sample-1)) over the last axis, eq. ergodic."""
    samples = np.asarray(samples, dtype=np.float64)
    ns = samples.shape[-1]
    mean = np.sum(samples, axis=-1) / ns
    std = np.sqrt(np.sum((samples - mean[..., None]) ** 2, axis=-1) / (ns - 1))
    return mean, std


def dense_posterior(G, ML, y_obs, sigma):
    """C_post and mu_post of Appendix A with C^{-1} = M_L."""
    H = G.T @ G / sigma ** 2 + np.diag(ML)
    C_post = np.linalg.inv(H)
    mu = C_post @ (G.T @ np.ravel(y_obs)) / sigma ** 2
    return C_post, mu


def exact_sample(G, ML, y_obs, sigma, eta, xi):
    """Closed-form RTO sample of Appendix A for one draw (eta, xi), by a dense solve."""
    H = G.T @ G / sigma ** 2 + np.diag(ML)
    p_prior = xi / np.sqrt(ML)
    rhs = G.T @ np.ravel(y_obs) / sigma ** 2 + G.T @ np.ravel(eta) / sigma + ML * p_prior
    return np.linalg.solve(H, rhs)
