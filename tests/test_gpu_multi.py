"""Uneven batches: several meshes and sample counts in one grouped solve.

The grouped launches run the same per-row arithmetic as separate solves, so
the results must be bit-identical to one pat_rto_sample call per job; the
per-job results are in turn checked against the oracle for a few iterations.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import rto
from problems import as_precision, cube_problem, rel_l2

pytestmark = pytest.mark.gpu


def job(n, n_steps, n_obs, K, noise, seed):
    from paper_2607_21373_b300 import Mesh
    P = cube_problem(n, n_obs, n_steps, faces=S.LIMITED_VIEW_FACES, seed=seed, phantom="blobs20+vessels",
                     noise=noise, data=True)
    m = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], n_steps, precision="f32")
    y = torch.tensor(as_precision(P["y_obs"], "f32"), dtype=torch.float32, device="cuda")
    return P, {"mesh": m, "y_obs": y, "sigma": P["sigma"], "K": K, "seed": seed}


def test_grouped_batch_equals_separate_solves():
    from paper_2607_21373_b300 import rto_sample_multi
    specs = [(4, 28, 12, 16, 0.01, 11), (6, 41, 20, 8, 0.02, 12), (8, 55, 32, 4, 0.03, 13)]
    jobs = [job(*s)[1] for s in specs]
    outs = rto_sample_multi(jobs, 4)
    for j, o in zip(jobs, outs):
        ref = j["mesh"].rto_sample(j["y_obs"], j["sigma"], j["K"], 4, seed=j["seed"])
        assert torch.equal(o["samples"], ref["samples"])
        assert torch.equal(o["mean"], ref["mean"]) and torch.equal(o["std"], ref["std"])


def test_grouped_batch_matches_oracle_first_iterations():
    from paper_2607_21373_b300 import rto_sample_multi
    from oracle import rng as orng
    specs = [(4, 28, 12, 8, 0.01, 21), (6, 41, 20, 4, 0.02, 22)]
    made = [job(*s) for s in specs]
    outs = rto_sample_multi([j for _, j in made], 2)
    for (P, j), o in zip(made, outs):
        K, nt, n_obs = j["K"], P["n_steps"], P["det"].shape[0]
        eta = orng.normals(j["seed"], 0, nt * n_obs, K).reshape(nt, n_obs, K)
        xi = orng.normals(j["seed"], 1, P["xyz"].shape[0], K)
        eta, xi = as_precision(eta, "f32"), as_precision(xi, "f32")
        X, _ = rto.rto_samples(P["ops"], P["dt"], nt, as_precision(P["y_obs"], "f32"), P["sigma"], eta, xi, 2)
        assert rel_l2(o["samples"].cpu().numpy(), X) < 2e-4


def test_uneven_batch_workload_shape():
    """Six cubes 16^3..58^3 cells with N_T = 1000 n/58, K = 256..8 and 1-4 % noise, one grouped
    solve (2 iterations here); every job's samples equal its separate solve."""
    from paper_2607_21373_b300 import rto_sample_multi
    jobs = []
    for w in S.UNEVEN:
        _, j = job(w.n, w.n_steps, w.n_obs, w.K, w.noise, w.seed)
        jobs.append(j)
    outs = rto_sample_multi(jobs, 2, samples=True)
    for j, o in zip(jobs[:2] + jobs[-1:], outs[:2] + outs[-1:]):
        ref = j["mesh"].rto_sample(j["y_obs"], j["sigma"], j["K"], 2, seed=j["seed"])
        assert torch.equal(o["samples"], ref["samples"])
