"""Sample-parallel RTO across processes (one GPU per rank).

RTO samples are independent (Section 5: every perturbed problem is solved on
its own), so ranks draw disjoint sample sets and never exchange data while
solving.  The one exchange is the pointwise posterior statistics of
eq. ergodic over all ranks' samples, combined here from each rank's count,
mean and std with two FP64 all-reduces (sums of K_r m_r, then of the
within-rank and between-rank squared deviations).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def sample_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's batch: disjoint counter streams per rank."""
    return (int(base_seed) * 1_000_003 + int(rank)) & 0xFFFFFFFFFFFFFFFF


def allreduce_moments(mean: torch.Tensor, std: torch.Tensor, K: int, group=None):
    """Global pointwise mean and std (1/(K_total - 1)) from per-rank statistics.

    mean, std: this rank's [N] float64 mean and std over its K samples (std may
    be None when K == 1).  Returns (mean, std, K_total) on every rank.
    """
    dev = mean.device
    k = torch.tensor([float(K)], dtype=torch.float64, device=dev)
    dist.all_reduce(k, group=group)
    k_tot = float(k.item())
    s1 = (mean.double() * K).clone()
    dist.all_reduce(s1, group=group)
    mu = s1 / k_tot
    m2 = (std.double() ** 2) * (K - 1) if (std is not None and K > 1) else torch.zeros_like(mu)
    m2 = m2 + K * (mean.double() - mu) ** 2
    dist.all_reduce(m2, group=group)
    return mu, torch.sqrt(m2 / (k_tot - 1)), int(round(k_tot))
