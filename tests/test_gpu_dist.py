"""The library side of sample parallelism, on one GPU: draws keyed by global
sample index (pat_mesh_set_first_sample) and the two-pass pooled statistics
(pat_rto_moments, pat_moments_finish).  Two "ranks" are two meshes in one
process; the sum across processes that an all-reduce performs is done here by
adding the ranks' [N] buffers."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import rto
from problems import cube_problem, rel_l2

pytestmark = pytest.mark.gpu


def test_ranks_draw_the_samples_of_one_run_and_pool_its_statistics():
    from paper_2607_21373_b300 import Mesh
    P = cube_problem(8, 32, 200, seed=1001, data=True)
    y = torch.tensor(P["y_obs"], dtype=torch.float64, device="cuda")
    sig, seed, k = P["sigma"], 99, 2

    def mesh(first):
        m = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], 200, precision="f64")
        m.set_first_sample(first)
        return m

    whole = mesh(0).rto_sample(y, sig, 16, k, seed=seed)
    ranks = [mesh(0), mesh(8)]
    parts = [r.rto_sample(y, sig, 8, k, seed=seed) for r in ranks]
    X = torch.cat([p["samples"] for p in parts], dim=1).cpu().numpy()
    # rank r's samples are columns 8r .. 8r+7 of the one-run batch
    assert rel_l2(X, whole["samples"].cpu().numpy()) < 1e-10
    # pooled statistics by the library's two passes
    s = ranks[0].rto_moments(8) + ranks[1].rto_moments(8)
    mean = ranks[0].moments_finish(s, 16, 0)
    q = ranks[0].rto_moments(8, center=mean) + ranks[1].rto_moments(8, center=mean)
    std = ranks[0].moments_finish(q, 16, 1)
    mo, so = rto.ergodic_mean_std(X)
    assert rel_l2(mean.cpu().numpy(), mo) < 1e-14
    assert rel_l2(std.cpu().numpy(), so) < 1e-13
    assert rel_l2(std.cpu().numpy(), whole["std"].cpu().numpy()) < 1e-10


def test_first_sample_bounds():
    from paper_2607_21373_b300 import Mesh, PatError
    P = cube_problem(8, 32, 200, seed=1001)
    m = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], 200, precision="f32")
    m.set_first_sample((1 << 23) - 1024)
    with pytest.raises(PatError):
        m.set_first_sample((1 << 23) - 1023)
    with pytest.raises(PatError):
        m.set_first_sample(-1)
