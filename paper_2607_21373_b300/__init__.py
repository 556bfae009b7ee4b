"""B300-native photoacoustic RTO sampler: Python binding of libpat.so.

Argument marshalling only: every step of the forward map, its transpose and
the batched CGLS runs in the library's CUDA kernels.  PyTorch provides device
memory and the current stream.  There is no CPU fallback: without a CUDA
device or without libpat.so these calls raise.

    mesh = Mesh(xyz, tets, det_xyz, dt, n_steps, precision="f32")
    Y = mesh.forward(p0)                      # [N_T, N_obs(, K)]
    g = mesh.adjoint(Y)                       # [N(, K)]
    out = mesh.rto_sample(y_obs, sigma, K=64, n_iter=100)
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import PatError

__all__ = ["Mesh", "MaternPrior", "PatError", "draw_normals", "rto_sample_multi", "lib", "F32", "F64"]

F32, F64 = 0, 1
MESH_SKIP_STABILITY, MESH_KEEP_ZEROS, MESH_SINGLE_COEF, MESH_HOST_ONLY, MESH_TWO_LEVEL, MESH_NO_GRAPHS = (
    0x1, 0x2, 0x4, 0x8, 0x10, 0x20)


def lib():
    return _lib.load()


def _stream(device=None):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _f64c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Mesh:
    """Device copy of a P1 tetrahedral mesh's operators (pat_mesh_create)."""

    def __init__(self, xyz, tets, det_xyz, dt, n_steps, precision="f32", c2=None, flags=0):
        L = lib()
        self.host_only = bool(int(flags) & MESH_HOST_ONLY)
        if self.host_only:
            self.device = None          # assembly and exports only; compute calls raise
        elif not torch.cuda.is_available():
            raise RuntimeError("paper_2607_21373_b300 needs a CUDA device (no CPU fallback)")
        else:
            self.device = torch.device("cuda", torch.cuda.current_device())
        xyz = _f64c(xyz)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        det = _f64c(det_xyz)
        c2a = None if c2 is None else _f64c(c2)
        self.prec = F64 if precision in ("f64", F64) else F32
        self.dtype = torch.float64 if self.prec == F64 else torch.float32
        h = C.c_void_p()
        _lib.check(L.pat_mesh_create(
            xyz.ctypes.data, len(xyz), tets.ctypes.data, len(tets),
            None if c2a is None else c2a.ctypes.data, det.ctypes.data, len(det), float(dt), int(n_steps),
            self.prec, int(flags), C.byref(h)))
        self._h = h
        info = _lib.MeshInfo()
        _lib.check(L.pat_mesh_query(h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in _lib.MeshInfo._fields_}
        self.N = info.n_nodes
        self.n_obs = info.n_obs
        self.n_steps = info.n_steps
        self.dt = info.dt
        self._ws = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._LIB is not None:
            _lib._LIB.pat_mesh_destroy(h)
            self._h = None

    # -- host exports ------------------------------------------------------
    def export(self):
        """Lumped mass, sensor nodes and P1 weights (4 per sensor, unused ones with
        weight 0), boundary faces (host numpy)."""
        ml = np.empty(self.N)
        dn = np.empty((self.n_obs, 4), dtype=np.int32)
        dw = np.empty((self.n_obs, 4))
        bf = np.empty((self.info["n_boundary_faces"], 3), dtype=np.int32)
        _lib.check(lib().pat_mesh_export(self._h, ml.ctypes.data, dn.ctypes.data, dw.ctypes.data,
                                         bf.ctypes.data))
        return {"ML": ml, "det_nodes": dn, "det_w": dw, "bfaces": bf}

    def export_csr(self, which):
        """K (which=0, full graph) or B (which=1) as (row_ptr, col, val) host arrays."""
        L = lib()
        nnz = C.c_int64()
        _lib.check(L.pat_mesh_export_csr(self._h, which, C.byref(nnz), None, None, None))
        rp = np.empty(self.N + 1, dtype=np.int64)
        col = np.empty(nnz.value, dtype=np.int32)
        val = np.empty(nnz.value)
        _lib.check(L.pat_mesh_export_csr(self._h, which, C.byref(nnz), rp.ctypes.data, col.ctypes.data,
                                         val.ctypes.data))
        return rp, col, val

    # -- workspace ---------------------------------------------------------
    def workspace_bytes(self, op, K):
        b = C.c_size_t()
        _lib.check(lib().pat_workspace_bytes(self._h, op, K, C.byref(b)))
        return b.value

    def workspace(self, op, K):
        """A cached, 256-byte aligned device workspace for (op, K)."""
        key = (op, K)
        nb = self.workspace_bytes(op, K)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < nb + 256:
            ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
            self._ws[key] = ws
        off = (-ws.data_ptr()) % 256
        return ws[off:off + nb]

    def _check_field(self, t, shape, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous CUDA {self.dtype} tensor")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")

    # -- forward map and transpose -------------------------------------------
    def forward(self, p0, scale=1.0, out=None):
        """Y = scale * G p0; p0 [N] or [N, K] -> Y [N_T, N_obs] or [N_T, N_obs, K]."""
        K = 1 if p0.dim() == 1 else p0.shape[1]
        self._check_field(p0, (self.N,) if p0.dim() == 1 else (self.N, K), "p0")
        shape = (self.n_steps, self.n_obs) + (() if p0.dim() == 1 else (K,))
        if out is None:
            out = torch.empty(shape, dtype=self.dtype, device=self.device)
        self._check_field(out, shape, "Y")
        ws = self.workspace(0, K)
        _lib.check(lib().pat_forward(self._h, _ptr(p0), K, _ptr(out), float(scale), _ptr(ws), ws.numel(),
                                     _stream()))
        return out

    def adjoint(self, Yhat, scale=1.0, out=None):
        """p_hat = scale * G^T Yhat; Yhat [N_T, N_obs(, K)] -> [N(, K)]."""
        K = 1 if Yhat.dim() == 2 else Yhat.shape[2]
        self._check_field(Yhat, (self.n_steps, self.n_obs) + (() if Yhat.dim() == 2 else (K,)), "Yhat")
        shape = (self.N,) if Yhat.dim() == 2 else (self.N, K)
        if out is None:
            out = torch.empty(shape, dtype=self.dtype, device=self.device)
        self._check_field(out, shape, "p_hat")
        ws = self.workspace(1, K)
        _lib.check(lib().pat_adjoint(self._h, _ptr(Yhat), K, _ptr(out), float(scale), _ptr(ws), ws.numel(),
                                     _stream()))
        return out

    # -- RTO -------------------------------------------------------------
    def rto_sample(self, y_obs, sigma, K, n_iter, eta=None, xi=None, seed=0, samples=True, resid=False,
                   mean=True, stdev=None, solver="cgls"):
        """K RTO posterior samples by n_iter CGLS (pat_rto_sample) or LSQR
        (pat_rto_sample_lsqr) iterations.  With resid: CGLS gives the data and
        prior blocks of ||r_j||^2 per iterate, shape (n_iter + 1, K, 2); LSQR gives
        phibar_j^2 = ||r_j||^2, shape (n_iter + 1, K)."""
        if solver not in ("cgls", "lsqr"):
            raise ValueError("solver must be 'cgls' or 'lsqr'")
        self._check_field(y_obs, (self.n_steps, self.n_obs), "y_obs")
        if eta is not None:
            self._check_field(eta, (self.n_steps, self.n_obs, K), "eta")
        if xi is not None:
            self._check_field(xi, (self.N, K), "xi")
        stdev = (K >= 2) if stdev is None else stdev
        dev = self.device
        out = {}
        out["samples"] = torch.empty((self.N, K), dtype=torch.float64, device=dev) if samples else None
        out["mean"] = torch.empty(self.N, dtype=torch.float64, device=dev) if mean else None
        out["std"] = torch.empty(self.N, dtype=torch.float64, device=dev) if stdev else None
        rshape = (n_iter + 1, K, 2) if solver == "cgls" else (n_iter + 1, K)
        out["resid"] = torch.empty(rshape, dtype=torch.float64, device=dev) if resid else None
        ws = self.workspace(2, K)
        fn = lib().pat_rto_sample if solver == "cgls" else lib().pat_rto_sample_lsqr
        _lib.check(fn(
            self._h, _ptr(y_obs), float(sigma), K, n_iter, _ptr(eta), _ptr(xi), C.c_uint64(seed),
            _ptr(out["samples"]), _ptr(out["mean"]), _ptr(out["std"]), _ptr(out["resid"]), _ptr(ws),
            ws.numel(), _stream()))
        return out

    def map_estimate(self, y_obs, sigma, n_iter, solver="lsqr", resid=False):
        """MAP estimate (eq. MAP) by n_iter LSQR or CGLS iterations from zero
        (pat_map_estimate); returns x [N] float64 and, with resid, ||r_j||^2."""
        self._check_field(y_obs, (self.n_steps, self.n_obs), "y_obs")
        x = torch.empty(self.N, dtype=torch.float64, device=self.device)
        r = torch.empty(n_iter + 1, dtype=torch.float64, device=self.device) if resid else None
        ws = self.workspace(2, 1)
        _lib.check(lib().pat_map_estimate(self._h, _ptr(y_obs), float(sigma), n_iter,
                                          {"cgls": 0, "lsqr": 1}[solver], _ptr(x), _ptr(r), _ptr(ws), ws.numel(),
                                          _stream()))
        return (x, r) if resid else x

    def whitened_misfit(self, x, y_obs, sigma):
        """||G x_k - y_obs|| / (sigma sqrt(N_T N_obs)) per column of x [N] or [N, K]
        float64 (pat_whitened_misfit; the discrepancy-principle diagnostic)."""
        K = 1 if x.dim() == 1 else x.shape[1]
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise TypeError("x must be a contiguous CUDA float64 tensor")
        self._check_field(y_obs, (self.n_steps, self.n_obs), "y_obs")
        out = torch.empty(K, dtype=torch.float64, device=self.device)
        ws = self.workspace(2, K)
        _lib.check(lib().pat_whitened_misfit(self._h, _ptr(x), _ptr(y_obs), float(sigma), K, _ptr(out), _ptr(ws),
                                             ws.numel(), _stream()))
        return out

    def set_c2(self, c2):
        """Replace the per-tetrahedron squared sound speed (host or device array) and rebuild."""
        c2 = _f64c(c2.detach().cpu().numpy() if isinstance(c2, torch.Tensor) else c2)
        if c2.shape != (self.info["n_tets"],):
            raise ValueError(f"c2 must have shape ({self.info['n_tets']},)")
        _lib.check(lib().pat_mesh_set_c2(self._h, c2.ctypes.data))

    def grad_c2(self, p0, Yhat, want_p0_grad=True, out=None):
        """(dL/dc2 [n_tets] float64 summed over samples, G^T Yhat or None) for the misfit
        cotangent Yhat = dL/dY (pat_grad_c2).  out = (g, p0_grad or None) reuses output
        buffers: repeated calls on the same buffers replay one captured CUDA graph."""
        K = 1 if p0.dim() == 1 else p0.shape[1]
        self._check_field(p0, (self.N,) if p0.dim() == 1 else (self.N, K), "p0")
        self._check_field(Yhat, (self.n_steps, self.n_obs) + (() if p0.dim() == 1 else (K,)), "Yhat")
        if out is not None:
            g, pg = out
            if not (isinstance(g, torch.Tensor) and g.is_cuda and g.dtype == torch.float64 and g.is_contiguous()
                    and tuple(g.shape) == (self.info["n_tets"],)):
                raise TypeError("out[0] must be a contiguous CUDA float64 tensor of shape (n_tets,)")
            if pg is not None:
                self._check_field(pg, tuple(p0.shape), "out[1]")
        else:
            g = torch.empty(self.info["n_tets"], dtype=torch.float64, device=self.device)
            pg = torch.empty_like(p0) if want_p0_grad else None
        ws = self.workspace(3, K)
        _lib.check(lib().pat_grad_c2(self._h, _ptr(p0), _ptr(Yhat), K, _ptr(g), _ptr(pg), _ptr(ws), ws.numel(),
                                     _stream()))
        return g, pg

    def autotune(self, K, n_probe=20):
        """Time every step-kernel variant for K samples and keep the fastest (pat_autotune).
        Returns the timing table as a list of dicts."""
        ws = self.workspace(2, K)
        table = (_lib.TuneEntry * 256)()
        n = C.c_int32()
        _lib.check(lib().pat_autotune(self._h, K, _ptr(ws), ws.numel(), int(n_probe), table, C.byref(n),
                                      _stream()))
        return [{"direction": ("fwd", "adj")[e.direction], "V": e.V, "staged": bool(e.staged),
                 "packed": int(e.packed), "chunk": e.chunk, "min_blocks": e.min_blocks,
                 "early": bool(e.early), "zorder": bool(e.zorder), "big_blocks": bool(e.big_blocks),
                 "prefetch": e.prefetch, "persistent": int(e.persistent), "pdl": bool(e.pdl),
                 "wide_loads": bool(e.wide_loads), "l2_hints": bool(e.l2_hints), "gather_batch": int(e.gather_batch),
                 "tail_serial": bool(e.tail_serial), "own_async": int(e.own_async),
                 "prefetch_meta": bool(e.prefetch_meta), "dyn_chunks": bool(e.dyn_chunks),
                 "us_per_step": e.us_per_step}
                for e in table[:min(n.value, 256)]]

    def select_variant(self, K, direction, V, packed=1, chunk=4, staged=False, min_blocks=1, early=False,
                       zorder=False, big_blocks=False, prefetch=0, persistent=False, pdl=False, wide_loads=False,
                       l2_hints=False, gather_batch=0, tail_serial=False, own_async=False,
                       prefetch_meta=False, dyn_chunks=False):
        """Force a step-kernel variant (pat_select_variant); direction 'fwd' or 'adj'."""
        e = _lib.TuneEntry(0 if direction == "fwd" else 1, V, int(staged), int(packed), int(chunk), int(min_blocks),
                           int(early), int(zorder), int(big_blocks), int(prefetch), int(persistent),
                           int(pdl), int(wide_loads), int(l2_hints), int(gather_batch), int(tail_serial),
                           int(own_async), int(prefetch_meta), int(dyn_chunks), 0.0)
        _lib.check(lib().pat_select_variant(self._h, K, 0 if direction == "fwd" else 1, C.byref(e)))

    def profile_enable(self, on=True):
        """Start (and reset) or stop live loop timing and launch counting."""
        _lib.check(lib().pat_profile_enable(self._h, int(bool(on))))

    def profile_read(self):
        """Synchronise and return the loop timings and launch counts since enable."""
        p = _lib.Profile()
        _lib.check(lib().pat_profile_read(self._h, C.byref(p)))
        return {k: getattr(p, k) for k, _ in _lib.Profile._fields_}

    def set_wait_cycles(self, cycles):
        """Copy-wait budget of the tile-staged step kernels in SM cycles (<= 0: the
        default); a tiny budget exercises the PAT_ETIMEOUT path (pat_mesh_set_wait_cycles)."""
        _lib.check(lib().pat_mesh_set_wait_cycles(self._h, int(cycles)))

    def set_first_sample(self, first):
        """Library-drawn perturbations of sample k use the draw index first + k
        (pat_mesh_set_first_sample): rank r of a sample-parallel run sets r * K."""
        _lib.check(lib().pat_mesh_set_first_sample(self._h, int(first)))

    def rto_moments(self, K, center=None):
        """Sum over the K samples of the last solve held in the workspace of x
        (center None) or of (x - center)^2, [N] float64 (pat_rto_moments)."""
        out = torch.empty(self.N, dtype=torch.float64, device=self.device)
        ws = self.workspace(2, K)
        _lib.check(lib().pat_rto_moments(self._h, K, _ptr(center), _ptr(out), _ptr(ws), ws.numel(), _stream()))
        return out

    def moments_finish(self, v, n_samples, which):
        """In place: which 0, v / n (mean); which 1, sqrt(v / (n - 1)) (std) (pat_moments_finish)."""
        _lib.check(lib().pat_moments_finish(v.numel(), float(n_samples), int(which), _ptr(v), _stream()))
        return v

    def status(self, K):
        ws = self.workspace(2, K)
        _lib.check(lib().pat_rto_status(self._h, K, _ptr(ws), _stream()))

    # stepwise CGLS with access to the state (pat_cgls_*)
    def cgls_begin(self, y_obs, sigma, K, eta=None, xi=None, seed=0):
        ws = self.workspace(2, K)
        _lib.check(lib().pat_cgls_begin(self._h, _ptr(y_obs), float(sigma), K, _ptr(eta), _ptr(xi),
                                        C.c_uint64(seed), _ptr(ws), ws.numel(), _stream()))

    def lsqr_begin(self, y_obs, sigma, K, eta=None, xi=None, seed=0):
        ws = self.workspace(2, K)
        _lib.check(lib().pat_lsqr_begin(self._h, _ptr(y_obs), float(sigma), K, _ptr(eta), _ptr(xi),
                                        C.c_uint64(seed), _ptr(ws), ws.numel(), _stream()))

    def lsqr_iterate(self, sigma, K, n_iter, resid=None):
        ws = self.workspace(2, K)
        _lib.check(lib().pat_lsqr_iterate(self._h, float(sigma), K, n_iter, _ptr(resid), _ptr(ws), ws.numel(),
                                          _stream()))

    def lsqr_state(self, K):
        """Views of the LSQR state in the workspace: x, ub_d, ub_p (beta u), v, w,
        alpha, beta, rhobar, phibar [K], status."""
        off = (C.c_size_t * 7)()
        _lib.check(lib().pat_lsqr_layout(self._h, K, off))
        ws = self.workspace(2, K)
        N, D = self.N, self.n_steps * self.n_obs

        def view(o, n, dtype, shape):
            return ws[o:o + n * (8 if dtype == torch.float64 else 4)].view(dtype).view(shape)

        lsq = view(off[5], 12 * K, torch.float64, (12, K))
        return {"x": view(off[0], N * K, torch.float64, (N, K)),
                "ub_d": view(off[1], D * K, self.dtype, (self.n_steps, self.n_obs, K)),
                "ub_p": view(off[2], N * K, self.dtype, (N, K)),
                "v": view(off[3], N * K, self.dtype, (N, K)), "w": view(off[4], N * K, self.dtype, (N, K)),
                "alpha": lsq[0], "beta": lsq[1], "rhobar": lsq[2], "phibar": lsq[3],
                "status": ws[off[6]:off[6] + 4].view(torch.int32)}

    def cgls_iterate(self, sigma, K, n_iter, resid=None):
        ws = self.workspace(2, K)
        _lib.check(lib().pat_cgls_iterate(self._h, float(sigma), K, n_iter, _ptr(resid), _ptr(ws), ws.numel(),
                                          _stream()))

    def cgls_state(self, K):
        """Views of the CGLS state in the workspace: x, d, r_d, r_p, s, gamma, status."""
        off = (C.c_size_t * 7)()
        _lib.check(lib().pat_cgls_layout(self._h, K, off))
        ws = self.workspace(2, K)
        N, D = self.N, self.n_steps * self.n_obs
        rs = 8 if self.prec == F64 else 4

        def view(o, n, dtype, shape):
            return ws[o:o + n * (8 if dtype == torch.float64 else 4)].view(dtype).view(shape)

        return {
            "x": view(off[0], N * K, torch.float64, (N, K)),
            "d": view(off[1], N * K, self.dtype, (N, K)),
            "r_d": view(off[2], D * K, self.dtype, (self.n_steps, self.n_obs, K)),
            "r_p": view(off[3], N * K, self.dtype, (N, K)),
            "s": view(off[4], N * K, self.dtype, (N, K)),
            "gamma": view(off[5], K, torch.float64, (K,)),
            "status": ws[off[6]:off[6] + 4].view(torch.int32),
        }


class MaternPrior:
    """Whittle-Matern prior on a periodic box grid of n_grid^3 points carried to
    the nodes of an FP32 mesh (pat_matern_create), and RTO in its latent space."""

    def __init__(self, mesh, n_grid, box_lo, box_len, ell, s, sigma):
        lo = _f64c(box_lo)
        h = C.c_void_p()
        _lib.check(lib().pat_matern_create(mesh._h, int(n_grid), lo.ctypes.data, float(box_len), float(ell),
                                           float(s), float(sigma), C.byref(h)))
        self._h, self.mesh, self.n_grid = h, mesh, int(n_grid)
        self.G = self.n_grid ** 3
        self._ws = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._LIB is not None:
            _lib._LIB.pat_matern_destroy(h)
            self._h = None

    def workspace(self, K):
        nb = C.c_size_t()
        _lib.check(lib().pat_matern_workspace_bytes(self.mesh._h, self._h, K, C.byref(nb)))
        ws = self._ws.get(K)
        if ws is None or ws.numel() < nb.value + 256:
            ws = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.mesh.device)
            self._ws[K] = ws
        off = (-ws.data_ptr()) % 256
        return ws[off:off + nb.value]

    def apply(self, op, field):
        """op "T" (grid -> grid), "P" (grid -> nodes), "PT" (nodes -> grid) or
        "PT_T" = P T (grid -> nodes) on a float32 CUDA field [points, K]."""
        code = {"T": 0, "P": 1, "PT": 2, "PT_T": 3}[op]
        K = field.shape[1]
        rows = self.mesh.N if code in (1, 3) else self.G
        out = torch.empty((rows, K), dtype=torch.float32, device=field.device)
        ws = self.workspace(K)
        _lib.check(lib().pat_matern_apply(self.mesh._h, self._h, code, _ptr(field), K, _ptr(out), _ptr(ws),
                                          ws.numel(), _stream()))
        return out

    def rto_sample(self, y_obs, sigma, K, n_iter, eta=None, xi=None, seed=0, latent=False, samples=True,
                   mean=True, stdev=None):
        """K latent-space RTO samples (pat_rto_sample_matern): nodal samples
        P T z [N, K] float64, their mean and std, and with latent the z [G, K]."""
        m = self.mesh
        stdev = (K >= 2) if stdev is None else stdev
        dev = m.device
        out = {"z": torch.empty((self.G, K), dtype=torch.float64, device=dev) if latent else None,
               "samples": torch.empty((m.N, K), dtype=torch.float64, device=dev) if samples else None,
               "mean": torch.empty(m.N, dtype=torch.float64, device=dev) if mean else None,
               "std": torch.empty(m.N, dtype=torch.float64, device=dev) if stdev else None}
        ws = self.workspace(K)
        _lib.check(lib().pat_rto_sample_matern(
            m._h, self._h, _ptr(y_obs), float(sigma), K, int(n_iter), _ptr(eta), _ptr(xi), C.c_uint64(seed),
            _ptr(out["z"]), _ptr(out["samples"]), _ptr(out["mean"]), _ptr(out["std"]), _ptr(ws), ws.numel(),
            _stream()))
        return out

    def status(self, K):
        ws = self.workspace(K)
        _lib.check(lib().pat_rto_status(self.mesh._h, K, _ptr(ws), _stream()))

    def state(self, K):
        """Views of the latent CGLS state left in the workspace by rto_sample
        (pat_matern_layout): z, d, r_p (latent residual), s, gamma, r_d, status."""
        off = (C.c_size_t * 7)()
        _lib.check(lib().pat_matern_layout(self.mesh._h, self._h, K, off))
        ws = self.workspace(K)
        m, G = self.mesh, self.G

        def view(o, n, dtype, shape):
            return ws[o:o + n * (8 if dtype == torch.float64 else 4)].view(dtype).view(shape)

        return {"z": view(off[0], G * K, torch.float64, (G, K)), "d": view(off[1], G * K, torch.float32, (G, K)),
                "r_p": view(off[2], G * K, torch.float32, (G, K)), "s": view(off[3], G * K, torch.float32, (G, K)),
                "gamma": view(off[4], K, torch.float64, (K,)),
                "r_d": view(off[5], m.n_steps * m.n_obs * K, torch.float32, (m.n_steps, m.n_obs, K)),
                "status": ws[off[6]:off[6] + 4].view(torch.int32)}


def rto_sample_multi(jobs, n_iter, samples=True):
    """Uneven batch (pat_rto_sample_multi): ``jobs`` is a list of dicts with keys
    mesh, y_obs, sigma, K and optionally eta, xi, seed.  Returns one output dict
    per job (samples, mean, std) as in Mesh.rto_sample."""
    arr = (_lib.RtoJob * len(jobs))()
    outs, keep = [], []
    for q, j in zip(arr, jobs):
        m, K = j["mesh"], j["K"]
        m._check_field(j["y_obs"], (m.n_steps, m.n_obs), "y_obs")
        dev = m.device
        o = {"samples": torch.empty((m.N, K), dtype=torch.float64, device=dev) if samples else None,
             "mean": torch.empty(m.N, dtype=torch.float64, device=dev),
             "std": torch.empty(m.N, dtype=torch.float64, device=dev) if K >= 2 else None}
        ws = m.workspace(2, K)
        q.mesh, q.y_obs, q.sigma, q.K = m._h.value, j["y_obs"].data_ptr(), float(j["sigma"]), K
        q.eta = 0 if j.get("eta") is None else j["eta"].data_ptr()
        q.xi = 0 if j.get("xi") is None else j["xi"].data_ptr()
        q.seed = int(j.get("seed", 0))
        q.samples = 0 if o["samples"] is None else o["samples"].data_ptr()
        q.mean = o["mean"].data_ptr()
        q.stdev = 0 if o["std"] is None else o["std"].data_ptr()
        q.workspace, q.workspace_bytes = ws.data_ptr(), ws.numel()
        outs.append(o)
        keep.append(ws)
    _lib.check(lib().pat_rto_sample_multi(len(jobs), arr, int(n_iter), _stream()))
    return outs


def draw_normals(seed, stream_id, n_elem, K, device=None):
    """The library's counter-based N(0,1) draws (pat_draw_normals), [n_elem, K] float64."""
    out = torch.empty((n_elem, K), dtype=torch.float64, device=device or "cuda")
    _lib.check(lib().pat_draw_normals(C.c_uint64(seed), stream_id, n_elem, K, _ptr(out), _stream()))
    return out
