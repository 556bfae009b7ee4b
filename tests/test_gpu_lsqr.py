"""GPU parity of the batched LSQR driver, the MAP estimate and the discrepancy
diagnostic against the FP64 oracle (oracle/rto.py: lsqr, map_estimate,
whitened_misfit, pinned in tests/test_oracle_rto.py).

As for CGLS, Krylov iterates amplify rounding once Ritz values converge, so
parity is checked (1) elementwise for the first iterations, (2) per iteration
at any depth as one oracle LSQR step from the GPU's own state, and (3) against
the closed forms of Appendix A at convergence.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import rng as orng
from oracle import rto, wave
from problems import as_precision, cube_problem, rel_l2

pytestmark = pytest.mark.gpu


def dev(a, prec):
    return torch.tensor(np.asarray(a), dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda")


def setup(prec, n=8, n_obs=32, n_steps=200, K=4, seed=1001):
    from paper_2607_21373_b300 import Mesh
    P = cube_problem(n, n_obs, n_steps, seed=seed, data=True)
    m = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], n_steps, precision=prec)
    N = P["xyz"].shape[0]
    y = as_precision(P["y_obs"], prec)
    eta = as_precision(S.standard_normal((n_steps, n_obs, K), seed + 15), prec)
    xi = as_precision(S.standard_normal((N, K), seed + 16), prec)
    return P, m, y, eta, xi


@pytest.mark.parametrize("prec,K,k,tol", [("f64", 8, 3, 1e-9), ("f64", 1, 2, 1e-10), ("f32", 4, 2, 2e-4),
                                          ("f32", 16, 1, 2e-5)])
def test_first_lsqr_iterations_match_oracle(prec, K, k, tol):
    P, m, y, eta, xi = setup(prec, K=K)
    out = m.rto_sample(dev(y, prec), P["sigma"], K, k, eta=dev(eta, prec), xi=dev(xi, prec), resid=True,
                       solver="lsqr")
    X, hist = rto.rto_samples_lsqr(P["ops"], P["dt"], P["n_steps"], y, P["sigma"], eta, xi, k)
    assert rel_l2(out["samples"].cpu().numpy(), X) < tol
    assert rel_l2(out["resid"].cpu().numpy(), hist ** 2) < tol        # ||r_j||^2 = phibar^2


@pytest.mark.parametrize("prec,K,depth,tol", [("f64", 4, 25, 1e-9), ("f32", 4, 25, 2e-4), ("f32", 64, 4, 2e-4)])
def test_each_lsqr_iteration_matches_one_oracle_step(prec, K, depth, tol):
    """From the GPU's LSQR state after `depth` iterations (u = ub / beta), one
    oracle LSQR step equals the GPU's next state."""
    P, m, y, eta, xi = setup(prec, K=K)
    sig = P["sigma"]
    m.lsqr_begin(dev(y, prec), sig, K, eta=dev(eta, prec), xi=dev(xi, prec))
    m.lsqr_iterate(sig, K, depth)
    st = {k: v.clone() for k, v in m.lsqr_state(K).items()}
    beta = st["beta"].cpu().numpy()
    state = {"x": st["x"].cpu().numpy(), "v": st["v"].cpu().double().numpy(), "w": st["w"].cpu().double().numpy(),
             "u": (st["ub_d"].cpu().double().numpy() / beta, st["ub_p"].cpu().double().numpy() / beta),
             "alpha": st["alpha"].cpu().numpy(), "phibar": st["phibar"].cpu().numpy(),
             "rhobar": st["rhobar"].cpu().numpy()}
    A, AT = rto.extended_operator(P["ops"], P["dt"], P["n_steps"], sig)
    ref = rto.lsqr_step(A, AT, state, True)
    m.lsqr_iterate(sig, K, 1)
    nxt = m.lsqr_state(K)
    assert int(nxt["status"].item()) == 0
    b1 = nxt["beta"].cpu().numpy()
    assert rel_l2(nxt["x"].cpu().numpy(), ref["x"]) < tol
    assert rel_l2(nxt["v"].cpu().double().numpy(), ref["v"]) < tol
    assert rel_l2(nxt["w"].cpu().double().numpy(), ref["w"]) < tol
    assert rel_l2(nxt["ub_d"].cpu().double().numpy() / b1, ref["u"][0]) < tol
    assert rel_l2(nxt["ub_p"].cpu().double().numpy() / b1, ref["u"][1]) < tol
    for key in ("alpha", "phibar", "rhobar"):
        assert np.all(np.abs(nxt[key].cpu().numpy() - ref[key]) <= tol * np.abs(ref[key])), key


def test_lsqr_and_cgls_agree_while_rounding_is_small():
    P, m, y, eta, xi = setup("f64", K=4)
    a = m.rto_sample(dev(y, "f64"), P["sigma"], 4, 3, eta=dev(eta, "f64"), xi=dev(xi, "f64"), solver="lsqr")
    b = m.rto_sample(dev(y, "f64"), P["sigma"], 4, 3, eta=dev(eta, "f64"), xi=dev(xi, "f64"), solver="cgls")
    assert rel_l2(a["samples"].cpu().numpy(), b["samples"].cpu().numpy()) < 1e-9


@pytest.mark.parametrize("prec,tol", [("f64", 1e-8), ("f32", 1e-3)])
def test_converged_lsqr_samples_and_map_are_the_closed_forms(prec, tol):
    """Appendix A: the converged sample C_post[G^T y/s^2 + G^T eta/s + M_L p_prior];
    with zero perturbations (eq. MAP) the posterior mean mu_post."""
    P, m, y, eta, xi = setup(prec, n=2, n_obs=8, n_steps=30, K=3, seed=11)
    G = wave.forward_matrix_dense(P["ops"], P["dt"], P["n_steps"])
    out = m.rto_sample(dev(y, prec), P["sigma"], 3, 300, eta=dev(eta, prec), xi=dev(xi, prec), solver="lsqr")
    X = out["samples"].cpu().numpy()
    for k in range(3):
        ref = rto.exact_sample(G, P["ops"]["ML"], y, P["sigma"], eta[..., k], xi[:, k])
        assert rel_l2(X[:, k], ref) < tol
    _, mu = rto.dense_posterior(G, P["ops"]["ML"], y, P["sigma"])
    for solver in ("lsqr", "cgls"):
        x, r = m.map_estimate(dev(y, prec), P["sigma"], 300, solver=solver, resid=True)
        assert rel_l2(x.cpu().numpy(), mu) < tol
        r = r.cpu().numpy()
        assert r[-1] <= r[0] and np.all(np.isfinite(r))


def test_map_first_iterations_match_oracle():
    P, m, y, eta, xi = setup("f64")
    for solver in ("lsqr", "cgls"):
        x, r = m.map_estimate(dev(y, "f64"), P["sigma"], 3, solver=solver, resid=True)
        xo, ho = rto.map_estimate(P["ops"], P["dt"], P["n_steps"], y, P["sigma"], 3, solver)
        assert rel_l2(x.cpu().numpy(), xo) < 1e-9
        assert rel_l2(r.cpu().numpy(), ho ** 2 if solver == "lsqr" else ho) < 1e-9


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_whitened_misfit_matches_oracle(prec, tol):
    P, m, y, eta, xi = setup(prec, K=3)
    X = np.stack([P["p0"], 0.5 * P["p0"], np.zeros_like(P["p0"])], axis=1)
    X = as_precision(X, prec)
    got = m.whitened_misfit(torch.tensor(X, dtype=torch.float64, device="cuda"), dev(y, prec), P["sigma"])
    ref = rto.whitened_misfit(P["ops"], P["dt"], P["n_steps"], X, y, P["sigma"])
    assert np.all(np.abs(got.cpu().numpy() - ref) <= tol * np.abs(ref))


def test_stepwise_lsqr_equals_one_call_and_seeded_draws():
    P, m, y, eta, xi = setup("f32", K=4)
    sig = P["sigma"]
    one = m.rto_sample(dev(y, "f32"), sig, 4, 5, seed=9, solver="lsqr")["samples"].clone()
    m.lsqr_begin(dev(y, "f32"), sig, 4, seed=9)
    m.lsqr_iterate(sig, 4, 3)
    m.lsqr_iterate(sig, 4, 2)
    assert torch.equal(m.lsqr_state(4)["x"], one)
    N = P["xyz"].shape[0]
    e = orng.normals(9, 0, P["n_steps"] * 32, 4).reshape(P["n_steps"], 32, 4)
    x = orng.normals(9, 1, N, 4)
    # device draws are added to y / sigma before rounding, passed ones after: the
    # first-iteration difference is FP32 rounding, which the Krylov recurrences
    # then amplify (~1e5 by iteration 5 on this mesh), so compare early
    a = m.rto_sample(dev(y, "f32"), sig, 4, 2, seed=9, solver="lsqr")["samples"]
    b = m.rto_sample(dev(y, "f32"), sig, 4, 2, eta=dev(e, "f32"), xi=dev(x, "f32"), solver="lsqr")["samples"]
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-5


def test_lsqr_bad_arguments_and_nonfinite_data():
    from paper_2607_21373_b300 import PatError
    P, m, y, eta, xi = setup("f32", K=2)
    with pytest.raises(PatError, match="PAT_EINVAL"):
        m.rto_sample(dev(y, "f32"), -1.0, 2, 3, solver="lsqr")
    with pytest.raises(PatError, match="PAT_EINVAL"):
        m.rto_sample(dev(y, "f32"), P["sigma"], 1, 3, stdev=True, solver="lsqr")
    out = m.rto_sample(dev(y, "f32"), P["sigma"], 2, 0, eta=dev(eta, "f32"), xi=dev(xi, "f32"), solver="lsqr")
    assert torch.count_nonzero(out["samples"]) == 0
    y = y.copy()
    y[3, 4] = np.nan
    m.rto_sample(dev(y, "f32"), P["sigma"], 2, 2, eta=dev(eta, "f32"), xi=dev(xi, "f32"), solver="lsqr")
    with pytest.raises(PatError, match="PAT_ENUMERIC"):
        m.status(2)
