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


def job_flags(n, n_steps, n_obs, K, noise, seed, flags):
    from paper_2607_21373_b300 import Mesh
    P = cube_problem(n, n_obs, n_steps, faces=S.LIMITED_VIEW_FACES, seed=seed, phantom="blobs20+vessels",
                     noise=noise, data=True)
    m = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], n_steps, precision="f32", flags=flags)
    y = torch.tensor(as_precision(P["y_obs"], "f32"), dtype=torch.float32, device="cuda")
    return P, {"mesh": m, "y_obs": y, "sigma": P["sigma"], "K": K, "seed": seed}


@pytest.mark.parametrize("keep_zeros", [False, True])
def test_persistent_grouped_batch_equals_separate_solves(keep_zeros):
    """K a multiple of 8 for every job: the grouped step launches are one
    persistent fixed-width grid over all jobs (8 slots on the pruned lattice, 16
    on the full graph), replayed from CUDA graphs; results equal separate solves
    bit for bit."""
    from paper_2607_21373_b300 import MESH_KEEP_ZEROS, rto_sample_multi
    flags = MESH_KEEP_ZEROS if keep_zeros else 0
    specs = [(4, 28, 12, 32, 0.01, 31), (6, 41, 20, 16, 0.02, 32), (9, 62, 40, 8, 0.03, 33)]
    jobs = [job_flags(*s, flags)[1] for s in specs]
    outs = rto_sample_multi(jobs, 5)
    for j, o in zip(jobs, outs):
        ref = j["mesh"].rto_sample(j["y_obs"], j["sigma"], j["K"], 5, seed=j["seed"])
        assert torch.equal(o["samples"], ref["samples"])
        assert torch.equal(o["mean"], ref["mean"]) and torch.equal(o["std"], ref["std"])


def test_persistent_grouped_batch_one_oracle_step_per_job():
    """After ten grouped CGLS iterations, one oracle step from each job's own
    GPU state equals that job's next state (the state stays in each job's
    workspace; one more grouped iteration advances every job)."""
    from paper_2607_21373_b300 import MESH_KEEP_ZEROS, rto_sample_multi
    specs = [(5, 34, 16, 16, 0.01, 41), (8, 55, 32, 8, 0.02, 42)]
    made = [job_flags(*s, MESH_KEEP_ZEROS) for s in specs]
    jobs = [j for _, j in made]
    rto_sample_multi(jobs, 10)
    refs = []
    for P, j in made:
        K, sig = j["K"], j["sigma"]
        st = {k: v.clone() for k, v in j["mesh"].cgls_state(K).items()}
        state = {"x": st["x"].cpu().double().numpy(), "d": st["d"].cpu().double().numpy(),
                 "r": (st["r_d"].cpu().double().numpy(), st["r_p"].cpu().double().numpy()),
                 "s": st["s"].cpu().double().numpy(), "gamma": st["gamma"].cpu().numpy()}
        A, AT = rto.extended_operator(P["ops"], P["dt"], P["n_steps"], sig)
        refs.append(rto.cgls_step(A, AT, state, True))
    # one more iteration of every job, continuing from the state in the workspaces
    for (P, j) in made:
        j["mesh"].cgls_iterate(j["sigma"], j["K"], 1)
    for (P, j), ref in zip(made, refs):
        nxt = j["mesh"].cgls_state(j["K"])
        assert int(nxt["status"].item()) == 0
        assert rel_l2(nxt["x"].cpu().numpy(), ref["x"]) < 1e-4
        assert rel_l2(nxt["d"].cpu().double().numpy(), ref["d"]) < 1e-4
        assert rel_l2(nxt["r_d"].cpu().double().numpy(), ref["r"][0]) < 1e-4
