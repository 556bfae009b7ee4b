"""Failure detection on the GPU without a fault: the tile-staged step kernels
and the 16-slot kernel with bulk-copied own rows wait for their bulk copies
with a bounded mbarrier wait, and a block (warp) whose wait runs out records
PAT_ETIMEOUT in the mesh's status word, waits for its copies in flight to land
and returns (carries on).  A budget of one SM cycle makes every such wait
run out (the copies themselves complete normally), so the timeout path runs
end to end; the host reads PAT_ETIMEOUT, and the same mesh then gives oracle
results with the default budget."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import rto
from problems import as_precision, cube_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [dict(V=8, packed=2), dict(V=8, packed=4)])
def test_copy_wait_timeout_is_reported_and_recovered(variant):
    from paper_2607_21373_b300 import Mesh, PatError
    P = cube_problem(8, 32, 200, seed=1001, data=True)
    K, k = 8, 2
    N = P["xyz"].shape[0]
    m = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], 200, precision="f32")
    for d in ("fwd", "adj"):
        m.select_variant(K, d, **variant)
    y = as_precision(P["y_obs"], "f32")
    eta = as_precision(S.standard_normal((200, 32, K), 61), "f32")
    xi = as_precision(S.standard_normal((N, K), 62), "f32")
    args = (torch.tensor(y, dtype=torch.float32, device="cuda"), P["sigma"], K, k)
    kw = dict(eta=torch.tensor(eta, dtype=torch.float32, device="cuda"),
              xi=torch.tensor(xi, dtype=torch.float32, device="cuda"))
    m.set_wait_cycles(1)
    m.rto_sample(*args, **kw)
    with pytest.raises(PatError, match="PAT_ETIMEOUT"):
        m.status(K)
    m.status(K)          # reported once, then clear
    m.set_wait_cycles(0)  # default budget
    out = m.rto_sample(*args, **kw)
    m.status(K)
    X, _ = rto.rto_samples(P["ops"], P["dt"], 200, y, P["sigma"], eta, xi, k)
    assert rel_l2(out["samples"].cpu().numpy(), X) < 2e-4


def test_own_row_copy_wait_timeout_on_the_full_graph():
    """The 16-slot row-major kernel whose warps copy their rows of x_s and
    x_{s-1} by bulk copies (own_async = 2), on the full P1 graph."""
    from paper_2607_21373_b300 import MESH_KEEP_ZEROS, Mesh, PatError
    P = cube_problem(8, 32, 200, seed=1001, data=True)
    K, k = 64, 2
    N = P["xyz"].shape[0]
    m = Mesh(P["xyz"], P["tets"], P["det"], P["dt"], 200, precision="f32", flags=MESH_KEEP_ZEROS)
    for d in ("fwd", "adj"):
        m.select_variant(K, d, V=8, packed=6, persistent=1, pdl=True, gather_batch=4, tail_serial=True,
                         own_async=2)
    y = as_precision(P["y_obs"], "f32")
    eta = as_precision(S.standard_normal((200, 32, K), 63), "f32")
    xi = as_precision(S.standard_normal((N, K), 64), "f32")
    args = (torch.tensor(y, dtype=torch.float32, device="cuda"), P["sigma"], K, k)
    kw = dict(eta=torch.tensor(eta, dtype=torch.float32, device="cuda"),
              xi=torch.tensor(xi, dtype=torch.float32, device="cuda"))
    m.set_wait_cycles(1)
    m.rto_sample(*args, **kw)
    with pytest.raises(PatError, match="PAT_ETIMEOUT"):
        m.status(K)
    m.status(K)
    m.set_wait_cycles(0)
    out = m.rto_sample(*args, **kw)
    m.status(K)
    X, _ = rto.rto_samples(P["ops"], P["dt"], 200, y, P["sigma"], eta, xi, k)
    assert rel_l2(out["samples"].cpu().numpy(), X) < 2e-4
