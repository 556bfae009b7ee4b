"""Sample-parallel statistics across ranks: world_size 2, gloo, CPU only.

The collective orchestration of paper_2607_21373_b300.dist runs here with the
library's two per-rank passes (sum of x, sum of squared deviations from a given
centre) and its finish step stood in by a small host object, since the library
itself needs a GPU; tests/test_gpu_dist.py checks those library calls."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


class HostMoments:
    """Test stand-in for a mesh's pat_rto_moments / pat_moments_finish over the
    samples X [N, K] this rank holds."""

    def __init__(self, X):
        self.X = torch.tensor(X, dtype=torch.float64)

    def rto_moments(self, K, center=None):
        assert K == self.X.shape[1]
        if center is None:
            return self.X.sum(dim=1)
        return ((self.X - center[:, None]) ** 2).sum(dim=1)

    def moments_finish(self, v, n, which):
        return v / n if which == 0 else torch.sqrt(v / (n - 1))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, X, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2607_21373_b300.dist import allreduce_moments
    parts = np.array_split(np.arange(X.shape[1]), world)
    mine = X[:, parts[rank]]
    mu, sd, kt = allreduce_moments(HostMoments(mine), mine.shape[1])
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


def test_first_samples_partition_the_global_indices():
    from paper_2607_21373_b300.dist import first_sample
    K, world = 64, 8
    idx = [first_sample(r, K) + k for r in range(world) for k in range(K)]
    assert sorted(idx) == list(range(K * world))
