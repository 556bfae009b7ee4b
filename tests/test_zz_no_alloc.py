"""pat_forward_noalloc: the forward map for callers that cannot allocate device memory.

Such callers (plug-ins whose host framework owns all device buffers, real-time
loops that must not allocate) pass only inputs and outputs; the time-stepping
state lives in a fixed array inside the library.  This file is collected last
so that a run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = a.double(), b.double()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_noalloc_forward_matches_forward_on_consecutive_calls():
    from paper_2607_21373_b300 import Mesh, _lib
    L = _lib.load()
    n, n_obs, nt, K = 8, 32, 200, 4
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, S.ALL_FACES, 31)
    mesh = Mesh(xyz, tets, det, 0.3 / n, nt, precision="f32")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):    # the second call reuses the array the first one left behind
        p0 = torch.tensor(S.standard_normal((len(xyz), K), 40 + call), dtype=torch.float32, device="cuda")
        ref = mesh.forward(p0)
        Y = torch.full((nt, n_obs, K), float("nan"), dtype=torch.float32, device="cuda")
        st = L.pat_forward_noalloc(mesh._h, C.c_void_p(p0.data_ptr()), K, C.c_void_p(Y.data_ptr()), 1.0, stream)
        assert st == 0, L.pat_last_error().decode()
        torch.cuda.synchronize()
        assert torch.isfinite(Y).all()
        # the same kernels on the same inputs as pat_forward (no atomics): the same bits,
        # so a partial read of a previous call's leftovers would show
        assert torch.equal(Y, ref)


def test_noalloc_forward_rejects_oversized_requests():
    from paper_2607_21373_b300 import Mesh, _lib
    L = _lib.load()
    n, nt = 8, 10
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(8, S.ALL_FACES, 32)
    mesh = Mesh(xyz, tets, det, 0.3 / n, nt, precision="f32")
    K = 1024                                     # 729 * 1024 > 524,288
    st = L.pat_forward_noalloc(mesh._h, C.c_void_p(256), K, C.c_void_p(256), 1.0, None)
    assert st == 1
    assert b"scratch array" in L.pat_last_error()


@pytest.mark.parametrize("precision,K,ok", [("f32", 1024, True), ("f64", 512, True), ("f64", 513, False)])
def test_noalloc_forward_at_the_size_limit(precision, K, ok):
    """N = 512 nodes (7^3 cells): N*K = 524,288 FP32 values (K = 1024) or 262,144
    FP64 values (K = 512) fill the 8 MiB array exactly and must run, giving
    pat_forward's result; one more FP64 sample (K = 513) must be refused."""
    from paper_2607_21373_b300 import Mesh, _lib
    L = _lib.load()
    n, n_obs, nt = 7, 16, 40
    xyz, tets = S.cube_mesh(n)
    assert len(xyz) == 512
    det = S.detector_points(n_obs, S.ALL_FACES, 33)
    mesh = Mesh(xyz, tets, det, 0.3 / n, nt, precision=precision)
    dt = torch.float32 if precision == "f32" else torch.float64
    p0 = torch.tensor(S.standard_normal((len(xyz), K), 50), dtype=dt, device="cuda")
    Y = torch.full((nt, n_obs, K), float("nan"), dtype=dt, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.pat_forward_noalloc(mesh._h, C.c_void_p(p0.data_ptr()), K, C.c_void_p(Y.data_ptr()), 1.0, stream)
    if not ok:
        assert st == 1 and b"scratch array" in L.pat_last_error()
        return
    assert st == 0, L.pat_last_error().decode()
    assert torch.equal(Y, mesh.forward(p0))
