"""Sample-parallel RTO across processes (one GPU per rank).

RTO samples are independent (Section 5: every perturbed problem is solved on
its own), so each rank solves its own K samples and never exchanges data while
solving; rank r's library draws are keyed by the global sample indices
r*K .. r*K + K - 1 (pat_mesh_set_first_sample), so the ranks together draw
exactly the perturbations of one K_total-sample run.  The one exchange is the
pointwise posterior statistics of eq. ergodic over all ranks' samples: the
library forms each rank's sums (pat_rto_moments) and finishes mean and std
(pat_moments_finish); this module only adds the [N] FP64 buffers across ranks
(two all-reduces, plus one of the sample count).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def first_sample(rank: int, K: int) -> int:
    """Global index of rank's first sample when every rank solves K samples."""
    return int(rank) * int(K)


def allreduce_moments(mesh, K: int, group=None):
    """Global pointwise mean and std (1/(K_total - 1)) of the samples of the last
    RTO solve of every rank on `mesh` (K samples on this rank), on every rank.
    Returns (mean, std, K_total); std is None when K_total < 2."""
    s = mesh.rto_moments(K)                        # sum_k x_ik over this rank's samples
    n = torch.tensor([float(K)], dtype=torch.float64, device=s.device)
    dist.all_reduce(n, group=group)
    dist.all_reduce(s, group=group)
    k_tot = float(n.item())
    mean = mesh.moments_finish(s, k_tot, 0)
    if k_tot < 2:
        return mean, None, int(round(k_tot))
    q = mesh.rto_moments(K, center=mean)           # sum_k (x_ik - mean_i)^2
    dist.all_reduce(q, group=group)
    return mean, mesh.moments_finish(q, k_tot, 1), int(round(k_tot))
