"""The Whittle-Matern prior on the GPU against the FP64 oracle (oracle/matern.py,
pinned by tests/test_oracle_matern.py): the spectral filter T, the trilinear
interpolation P and its transpose, and RTO in the latent space.

The unit-cube mesh [0, 1]^3 sits in the periodic box [-0.5, 1.5)^3; the
oracle's box is centred, so its nodes are the mesh's shifted by -0.5 (the same
grid points and weights).  FP32 fields: 1e-5 relative L2 for T, P, P^T; dot
test 1e-6; latent RTO elementwise for the first iterations at the FP32 RTO
tolerance of the other parity tests."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import matern, rto
from oracle import rng as orng
from problems import as_precision, cube_problem, rel_l2

pytestmark = pytest.mark.gpu

NG, ELL, SMOOTH, SIGMA = 16, 0.3, 1.5, 1.0


def setup(n=6, n_obs=16, n_steps=40, ng=NG):
    from paper_2607_21373_b300 import MaternPrior, Mesh
    P = cube_problem(n, n_obs, n_steps, seed=1010, data=True)
    m = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], n_steps, precision="f32")
    prior = MaternPrior(m, ng, (-0.5, -0.5, -0.5), 2.0, ELL, SMOOTH, SIGMA)
    filt = matern.spectral_filter(ng, 1.0, ELL, SMOOTH, SIGMA)
    idx, w = matern.trilinear(ng, 1.0, P["xyz"] - 0.5)
    return P, m, prior, filt, idx, w


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("ng,K", [(8, 2), (16, 8), (32, 3), (64, 32), (128, 4), (64, 5)])
def test_filter_T_matches_oracle(ng, K):
    """Every line length's four-step split (n_g = 8 .. 128: 1, 2, 4 or 8 threads
    per line and sample), sample chunks of 1 .. 16, even K (two samples per
    complex field) and odd K (real-input passes)."""
    P, m, prior, filt, idx, w = setup(ng=ng)
    z = as_precision(S.standard_normal((ng ** 3, K), 70 + K), "f32")
    out = prior.apply("T", dev(z)).cpu().numpy()
    ref = matern.apply_T(z.reshape(ng, ng, ng, K), filt).reshape(-1, K)
    assert rel_l2(out, ref) < 1e-5


def test_filter_T_largest_grid_matches_oracle():
    """n_g = 256 with 64 samples (32 complex pairs per chunk): 512-thread
    blocks and 64 KB of shared memory; two of the 64 columns against the oracle
    (T acts on each sample separately), and one sample alone (the unpacked
    real-input passes)."""
    ng, K = 256, 64
    P, m, prior, filt, idx, w = setup(ng=ng)
    z = S.device_standard_normal((ng ** 3, K), 77, "cuda")
    out = prior.apply("T", z)
    for c in (0, K - 1):
        zc = z[:, c].cpu().double().numpy()
        ref = matern.apply_T(zc.reshape(ng, ng, ng), filt).reshape(-1)
        assert rel_l2(out[:, c].cpu().numpy(), ref) < 1e-5
        one = prior.apply("T", z[:, c:c + 1].contiguous())
        assert rel_l2(one[:, 0].cpu().numpy(), ref) < 1e-5


def test_interpolation_and_transpose_match_oracle():
    P, m, prior, filt, idx, w = setup()
    K, G, N = 4, NG ** 3, P["xyz"].shape[0]
    g = as_precision(S.standard_normal((G, K), 80), "f32")
    v = as_precision(S.standard_normal((N, K), 81), "f32")
    Pg = prior.apply("P", dev(g))
    PTv = prior.apply("PT", dev(v))
    assert rel_l2(Pg.cpu().numpy(), matern.interp(g.reshape(NG, NG, NG, K), idx, w)) < 1e-6
    assert rel_l2(PTv.cpu().numpy(), matern.interp_T(v, idx, w, NG).reshape(G, K)) < 1e-6
    # P^T is P's transpose: <P g, v> = <g, P^T v>
    lhs = (Pg.double() * dev(v).double()).sum(dim=0)
    rhs = (dev(g).double() * PTv.double()).sum(dim=0)
    scale = Pg.double().norm(dim=0) * dev(v).double().norm(dim=0)
    assert torch.all((lhs - rhs).abs() <= 1e-6 * scale)
    # P T in one call
    PT = prior.apply("PT_T", dev(g)).cpu().numpy()
    ref = matern.interp(matern.apply_T(g.reshape(NG, NG, NG, K), filt), idx, w)
    assert rel_l2(PT, ref) < 1e-5


@pytest.mark.parametrize("k", [1, 2])
def test_latent_rto_first_iterations_match_oracle(k):
    P, m, prior, filt, idx, w = setup()
    K, G = 4, NG ** 3
    y = as_precision(P["y_obs"], "f32")
    eta = as_precision(S.standard_normal((P["n_steps"], 16, K), 90), "f32")
    xi = as_precision(S.standard_normal((G, K), 91), "f32")
    out = prior.rto_sample(dev(y), P["sigma"], K, k, eta=dev(eta), xi=dev(xi), latent=True)
    prior.status(K)
    z, p, _ = matern.latent_rto_samples(P["ops"], P["dt"], P["n_steps"], y, P["sigma"], eta,
                                        xi.reshape(NG, NG, NG, K), filt, idx, w, k, solver="cgls")
    assert rel_l2(out["z"].cpu().numpy(), z.reshape(G, K)) < 2e-4
    assert rel_l2(out["samples"].cpu().numpy(), p) < 2e-4
    mo, so = rto.ergodic_mean_std(out["samples"].cpu().numpy())
    assert rel_l2(out["mean"].cpu().numpy(), mo) < 1e-13
    assert rel_l2(out["std"].cpu().numpy(), so) < 1e-12


def test_latent_rto_one_oracle_step_from_the_gpu_state():
    """Deep iterations amplify rounding (the Krylov floor of the other parity
    tests), so the depth is checked one step at a time: the oracle's CGLS step
    from the GPU's latent state after 6 iterations against the GPU's state after
    7 (the solve is deterministic, so its first 6 iterations repeat bit for bit)."""
    P, m, prior, filt, idx, w = setup()
    K, G = 4, NG ** 3
    y = dev(as_precision(P["y_obs"], "f32"))
    eta = dev(as_precision(S.standard_normal((P["n_steps"], 16, K), 92), "f32"))
    xi = dev(as_precision(S.standard_normal((G, K), 93), "f32"))

    def run(k):
        prior.rto_sample(y, P["sigma"], K, k, eta=eta, xi=xi, latent=True, samples=False, mean=False,
                         stdev=False)
        prior.status(K)
        return {k_: v.clone() for k_, v in prior.state(K).items()}

    st, nxt = run(6), run(7)
    assert int(nxt["status"].item()) == 0
    grid = (NG, NG, NG, K)
    np64 = lambda t: t.cpu().double().numpy()
    state = {"x": np64(st["z"]).reshape(grid), "d": np64(st["d"]).reshape(grid),
             "r": (np64(st["r_d"]), np64(st["r_p"]).reshape(grid)), "s": np64(st["s"]).reshape(grid),
             "gamma": np64(st["gamma"])}
    A, AT = matern.latent_operator(P["ops"], P["dt"], P["n_steps"], P["sigma"], filt, idx, w)
    ref = rto.cgls_step(A, AT, state, True)
    assert rel_l2(np64(nxt["z"]), ref["x"].reshape(G, K)) < 1e-5
    assert rel_l2(np64(nxt["d"]), ref["d"].reshape(G, K)) < 1e-4
    assert rel_l2(np64(nxt["s"]), ref["s"].reshape(G, K)) < 1e-4
    assert rel_l2(np64(nxt["r_d"]), ref["r"][0]) < 1e-4
    assert rel_l2(np64(nxt["r_p"]), ref["r"][1].reshape(G, K)) < 1e-4
    g = np64(nxt["gamma"])
    assert np.all(np.abs(g - ref["gamma"]) <= 1e-4 * np.abs(ref["gamma"]))


def test_latent_rto_library_draws_are_the_published_generator():
    """NULL eta and xi: the library draws stream 0 (data) and stream 1 at the
    grid points (latent prior); the same draws regenerated by the oracle's
    generator and passed in give the same samples."""
    P, m, prior, filt, idx, w = setup()
    K, G, seed = 3, NG ** 3, 123
    y = dev(as_precision(P["y_obs"], "f32"))
    e = orng.normals(seed, 0, P["n_steps"] * 16, K).reshape(P["n_steps"], 16, K)
    x = orng.normals(seed, 1, G, K)
    a = prior.rto_sample(y, P["sigma"], K, 2, seed=seed, latent=True)["z"]
    b = prior.rto_sample(y, P["sigma"], K, 2, eta=dev(e), xi=dev(x), latent=True)["z"]
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-5


def test_matern_argument_errors():
    from paper_2607_21373_b300 import MaternPrior, Mesh, PatError
    P = cube_problem(6, 16, 40, seed=1010)
    m = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], 40, precision="f32")
    with pytest.raises(PatError, match="PAT_EINVAL"):
        MaternPrior(m, 24, (-0.5,) * 3, 2.0, ELL, SMOOTH, SIGMA)        # not a power of two
    with pytest.raises(PatError, match="PAT_EINVAL"):
        MaternPrior(m, 16, (0.2,) * 3, 2.0, ELL, SMOOTH, SIGMA)         # nodes outside the box
    m64 = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], 40, precision="f64")
    with pytest.raises(PatError, match="PAT_EUNSUPPORTED"):
        MaternPrior(m64, 16, (-0.5,) * 3, 2.0, ELL, SMOOTH, SIGMA)
