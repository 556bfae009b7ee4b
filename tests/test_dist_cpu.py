"""Sample-parallel statistics across ranks: world_size 2, gloo, CPU only."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, X, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2607_21373_b300.dist import allreduce_moments
    parts = np.array_split(np.arange(X.shape[1]), world)
    mine = torch.tensor(X[:, parts[rank]])
    K = mine.shape[1]
    m = mine.mean(dim=1)
    s = mine.std(dim=1, unbiased=True) if K > 1 else None
    mu, sd, kt = allreduce_moments(m, s, K)
    out[rank] = (mu.numpy(), sd.numpy(), kt)
    dist.destroy_process_group()


def test_allreduce_moments_equals_pooled_statistics():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((50, 7)) * 3 + 1
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), X, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        mu, sd, kt = out[r]
        assert kt == 7
        assert np.allclose(mu, X.mean(axis=1), rtol=0, atol=1e-13)
        assert np.allclose(sd, X.std(axis=1, ddof=1), rtol=1e-12, atol=0)


def test_sample_seeds_are_disjoint_per_rank():
    from paper_2607_21373_b300.dist import sample_seed
    assert len({sample_seed(5, r) for r in range(8)}) == 8
