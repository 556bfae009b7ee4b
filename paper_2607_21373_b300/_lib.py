"""ctypes declarations of libpat.so (the C ABI of include/pat.h)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

c_size_p = C.POINTER(C.c_size_t)


class MeshInfo(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int64), ("n_tets", C.c_int64), ("n_boundary_faces", C.c_int64),
        ("n_boundary_nodes", C.c_int64), ("nnz_K", C.c_int64), ("nnz_K_graph", C.c_int64),
        ("nnz_B", C.c_int64), ("n_obs", C.c_int32), ("n_steps", C.c_int32), ("prec", C.c_int32),
        ("dt", C.c_double), ("operator_bytes", C.c_double), ("tile_rows", C.c_int32),
        ("tile_max_staged", C.c_int32), ("tile_mean_staged", C.c_double),
    ]


class Profile(C.Structure):
    _fields_ = [("fwd_ms", C.c_double), ("adj_ms", C.c_double), ("fwd_loops", C.c_int64),
                ("adj_loops", C.c_int64), ("fwd_launches", C.c_int64), ("adj_launches", C.c_int64),
                ("total_launches", C.c_int64)]


class RtoJob(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("y_obs", C.c_void_p), ("sigma", C.c_double), ("K", C.c_int32),
                ("eta", C.c_void_p), ("xi", C.c_void_p), ("seed", C.c_uint64), ("samples", C.c_void_p),
                ("mean", C.c_void_p), ("stdev", C.c_void_p), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t)]


class TuneEntry(C.Structure):
    _fields_ = [("direction", C.c_int32), ("V", C.c_int32), ("staged", C.c_int32), ("packed", C.c_int32),
                ("chunk", C.c_int32), ("min_blocks", C.c_int32), ("early", C.c_int32), ("zorder", C.c_int32),
                ("big_blocks", C.c_int32), ("prefetch", C.c_int32), ("persistent", C.c_int32),
                ("pdl", C.c_int32), ("wide_loads", C.c_int32), ("l2_hints", C.c_int32), ("gather_batch", C.c_int32),
                ("tail_serial", C.c_int32), ("own_async", C.c_int32),
                ("prefetch_meta", C.c_int32), ("dyn_chunks", C.c_int32),
                ("us_per_step", C.c_double)]


# name -> (restype, argtypes); every compute call returns pat_status (int)
SIGNATURES = {
    "pat_mesh_create": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                  C.c_int32, C.c_double, C.c_int32, C.c_int, C.c_uint32,
                                  C.POINTER(C.c_void_p)]),
    "pat_mesh_destroy": (C.c_int, [C.c_void_p]),
    "pat_mesh_set_c2": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pat_grad_c2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_size_t, C.c_void_p]),
    "pat_mesh_query": (C.c_int, [C.c_void_p, C.POINTER(MeshInfo)]),
    "pat_mesh_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pat_mesh_export_csr": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "pat_workspace_bytes": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, c_size_p]),
    "pat_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_void_p,
                              C.c_size_t, C.c_void_p]),
    "pat_forward_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_void_p]),
    "pat_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_void_p,
                              C.c_size_t, C.c_void_p]),
    "pat_rto_sample": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_void_p,
                                 C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_size_t, C.c_void_p]),
    "pat_rto_sample_multi": (C.c_int, [C.c_int32, C.POINTER(RtoJob), C.c_int32, C.c_void_p]),
    "pat_rto_sample_lsqr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_size_t, C.c_void_p]),
    "pat_lsqr_begin": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_uint64, C.c_void_p, C.c_size_t, C.c_void_p]),
    "pat_lsqr_iterate": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                   C.c_size_t, C.c_void_p]),
    "pat_map_estimate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "pat_whitened_misfit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_size_t, C.c_void_p]),
    "pat_cgls_begin": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_uint64, C.c_void_p, C.c_size_t, C.c_void_p]),
    "pat_cgls_iterate": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                   C.c_size_t, C.c_void_p]),
    "pat_cgls_finish": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_size_t, C.c_void_p]),
    "pat_cgls_layout": (C.c_int, [C.c_void_p, C.c_int32, c_size_p]),
    "pat_lsqr_layout": (C.c_int, [C.c_void_p, C.c_int32, c_size_p]),
    "pat_rto_status": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "pat_mesh_set_wait_cycles": (C.c_int, [C.c_void_p, C.c_int64]),
    "pat_mesh_set_first_sample": (C.c_int, [C.c_void_p, C.c_int64]),
    "pat_rto_moments": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                  C.c_void_p]),
    "pat_moments_finish": (C.c_int, [C.c_int64, C.c_double, C.c_int32, C.c_void_p, C.c_void_p]),
    "pat_draw_normals": (C.c_int, [C.c_uint64, C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]),
    "pat_matern_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.POINTER(C.c_void_p)]),
    "pat_matern_destroy": (C.c_int, [C.c_void_p]),
    "pat_matern_layout": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, c_size_p]),
    "pat_matern_workspace_bytes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, c_size_p]),
    "pat_matern_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                   C.c_void_p, C.c_size_t, C.c_void_p]),
    "pat_rto_sample_matern": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_int32,
                                        C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "pat_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32, C.POINTER(TuneEntry),
                               C.POINTER(C.c_int32), C.c_void_p]),
    "pat_select_variant": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(TuneEntry)]),
    "pat_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "pat_profile_read": (C.c_int, [C.c_void_p, C.POINTER(Profile)]),
    "pat_last_error": (C.c_char_p, []),
    "pat_version": (C.c_char_p, []),
}

_LIB = None


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load (building first if needed) the in-tree libpat.so; raises if that fails."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libpat.so is missing at {path}; run paper_2607_21373_b300/build.py")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


STATUS = {0: "PAT_OK", 1: "PAT_EINVAL", 2: "PAT_ENOMEM", 3: "PAT_ECUDA", 4: "PAT_EUNSTABLE",
          5: "PAT_ENUMERIC", 6: "PAT_ETIMEOUT", 7: "PAT_EUNSUPPORTED"}


class PatError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int):
    if status != 0:
        raise PatError(status, _LIB.pat_last_error().decode())
