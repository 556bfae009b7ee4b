#!/usr/bin/env python
"""Throughput of the batched RTO sampler on B300 (one JSON line on stdout).

One step = one RTO batch: K posterior samples, each the CGLS solve of the
extended least-squares system with k iterations (2k+1 wave solves of N_T steps
per sample), on a seeded synthetic workload shaped like the paper's 3D problem
(Section 6.4: ~2e5 unknowns): unit cube 58^3 cells x 6 tets (205,379 nodes),
N_T = 1000, 1024 sensors on five faces, K = 64, k = 100, FP32 state with FP64
CGLS scalars.  The stiffness operator is the full P1 graph (15 entries per
interior row, the entries that cancel on the regular lattice kept, as on an
unstructured mesh); --mesh pruned drops those exact zeros, --mesh jitter moves
the interior nodes so that nothing cancels.  The timed region holds the whole
batch (data perturbations and prior draws come from the library's
counter-based generator on the device).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--mesh cube|pruned|jitter] [--tune-log FILE]

Under torchrun every rank runs its own K samples (sample parallelism, no data
collective; weak scaling); rank 0 prints the line.  --impl reference times the
FP64 CPU oracle on the same workload (a bounded, extrapolated sample, one
oracle process per host core).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as S  # noqa: E402

METRIC = "rto_samples_per_s"
UNIT = "samples/s"
MESH_KEEP_ZEROS = 0x2
MESH_TWO_LEVEL = 0x10
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one step launch of a
# kernel variant, from one ncu capture on the named workload (K = 64, 1024 sensors;
# profiles/step3w_persist_kernel_cube58_full_K64.md, step3e_persist_kernel_cube58_K64.md).  Used for the roofline's "traffic" only when the timed run uses that
# variant on that workload; null otherwise.
PROFILED_TRAFFIC = {
    ("cube", "step3w_persist_kernel<false> (16 slots row-major, rounds of 4, serial tail) (own rows async)"):
        180.555520e6,
    ("cube", "step3w_persist_kernel<false> (16 slots row-major, rounds of 4, columns per round, serial tail) "
             "(own rows async)"): 180.403968e6,
    ("cube", "step3w_persist_kernel<true> (16 slots row-major, rounds of 4) (own x_{s-1} rows async)"):
        181.347328e6,
    ("pruned", "step3e_persist_kernel<8,false> (256-thread blocks, PDL, L2 prefetch 1)"): 160.643584e6,
    ("pruned", "step3e_persist_kernel<8,true> (256-thread blocks, PDL, L2 prefetch 1)"): 159.604480e6,
    ("pruned", "step3e_persist_kernel<8,false> (1024-thread blocks, PDL)"): 159.210752e6,
    ("pruned", "step3e_persist_kernel<8,true> (1024-thread blocks, PDL)"): 158.733312e6,
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cells", type=int, default=58, help="cells per cube edge")
    ap.add_argument("--n-steps", type=int, default=1000)
    ap.add_argument("--n-obs", type=int, default=1024)
    ap.add_argument("--K", type=int, default=64)
    ap.add_argument("--k-iter", type=int, default=100)
    ap.add_argument("--order", default="native", choices=["native", "rcm", "morton"],
                    help="node numbering of the mesh handed to the library (reorder.py)")
    ap.add_argument("--mesh", default="cube", choices=["cube", "pruned", "jitter"],
                    help="cube: full P1 graph (default); pruned: exact-zero entries of the lattice dropped; "
                         "jitter: interior nodes moved by up to 0.15 h per axis (nothing cancels)")
    ap.add_argument("--plain-steps", type=int, default=3, help="timed K=1 samples (0: skip the plain form)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--cpu-procs", type=int, default=0, help="oracle processes (0: one per host core, at most 64)")
    ap.add_argument("--mesh-flags", type=int, default=0, help="extra pat_mesh_create flags (e.g. 16: two-level form)")
    ap.add_argument("--autotune", type=int, default=1, help="0: keep the library's default step-kernel variant")
    ap.add_argument("--tune-log", default="", help="write the autotuner's full timing table (JSON) to this file")
    ap.add_argument("--solver", default="cgls", choices=["cgls", "lsqr"],
                    help="least-squares solver of every RTO sample (the configured workload names CGLS)")
    ap.add_argument("--variant", default="", help="force a step-kernel variant for K (FWD or FWD,ADJ): "
                    + " | ".join(sorted(FORCED)))
    ap.add_argument("--workload", default="rto", choices=["rto", "uneven", "matern", "grad"],
                    help="rto: one mesh, K samples per batch (default); uneven: six cubes 16^3..58^3 cells with "
                         "K 256..8 and N_T 276..1000 in one grouped solve per step (k = 50); matern: the rto "
                         "workload with the Whittle-Matern prior (128^3 latent grid, l = 0.15, s = 1.5, sigma = 3); "
                         "grad: c2 and p0 gradients on a 32^3-cell cube, 1000 steps, K = 1 (sizes the options give "
                         "explicitly override these)")
    a = ap.parse_args(argv)
    given = sys.argv[1:] if argv is None else list(argv)
    for opt, attr in (("--cells", "cells_given"), ("--n-steps", "n_steps_given"), ("--n-obs", "n_obs_given"),
                      ("--K", "K_given")):
        setattr(a, attr, any(x == opt or x.startswith(opt + "=") for x in given))
    return a


# step-kernel variants that --variant can force (fields of pat_select_variant)
FORCED = {
    "tiled": dict(V=8, packed=2), "v8c2": dict(V=8, packed=1, chunk=2), "v4c4": dict(V=4, packed=1, chunk=4),
    "ell8": dict(V=8, packed=3), "ell4": dict(V=4, packed=3), "pipe": dict(V=8, packed=4),
    "ell8pp": dict(V=8, packed=3, persistent=1, pdl=True, prefetch=1),
    "ell8pb": dict(V=8, packed=3, persistent=1, pdl=True, big_blocks=True),
    "w16": dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4),
    "w16c": dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, early=True),
    "w16b8": dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=8),
    "w16b8c": dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=8, early=True),
    "w16big": dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, early=True, big_blocks=True),
    "w16cs": dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True),
    "w16r": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4),
    "w16rc": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True),
    "w16ro": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, tail_serial=True, own_async=True),
    "w16rb": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, tail_serial=True, own_async=2),
    "w16rcs": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True),
    "w16qop": dict(V=8, packed=5, persistent=1, pdl=True, gather_batch=4, tail_serial=True, own_async=True,
                   prefetch_meta=True),
    "w16rod": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, tail_serial=True, own_async=True,
                   dyn_chunks=True),
    "w16rcod": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True,
                    own_async=True, dyn_chunks=True),
    "w16rcop2": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, own_async=True),
    "w16rop2": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, own_async=True),
    "w16rco": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True,
                   own_async=True),
    "w16rop": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, tail_serial=True, own_async=True,
                   prefetch_meta=True),
    "w16rcox": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, early=True, tail_serial=True,
                    own_async=3),
    "w16rox": dict(V=8, packed=6, persistent=1, pdl=True, gather_batch=4, own_async=3),
    "e1": dict(V=1, packed=3),
    "g1": dict(V=1, packed=0),
    "pairs": dict(V=8, packed=7, persistent=1, pdl=True),
    "quads": dict(V=8, packed=8, persistent=1, pdl=True),
    "quadso": dict(V=8, packed=8, persistent=1, pdl=True, own_async=True),
    "pairs3": dict(V=8, packed=7, persistent=1, pdl=True, min_blocks=3),
}


def mesh_flags(a):
    return (0 if a.mesh == "pruned" else MESH_KEEP_ZEROS) | a.mesh_flags


def workload_config(a):
    w = S.BATCHED
    n = a.cells
    kind = {"cube": "Kuhn tets, full P1 graph (15 entries per interior row, lattice zeros kept)",
            "pruned": "Kuhn tets, exact-zero entries dropped (7-point interior rows)",
            "jitter": "Kuhn connectivity, interior nodes jittered by U[-0.15h, 0.15h]^3 (15 nonzeros per row)"}[a.mesh]
    return {
        "workload": f"cube{n}_rto_{a.mesh}: unit cube {n}^3 cells x 6 tets ({kind}), {(n + 1) ** 3} nodes, "
                    f"N_T={a.n_steps}, dt=0.3h, {a.n_obs} sensors on 5 faces, K={a.K} samples per batch, "
                    f"{a.solver.upper()} k={a.k_iter}, white-noise prior N(0, M_L^-1), 1% noise",
        "n_nodes": (n + 1) ** 3, "n_tets": 6 * n ** 3, "n_steps": a.n_steps, "n_obs": a.n_obs,
        "K": a.K, "solver": a.solver, "iters": a.k_iter, "noise": w.noise, "mesh": a.mesh,
        "node_steps_per_sample": (2 * a.k_iter + 1) * a.n_steps * (n + 1) ** 3,
        "l2": "inputs larger than L2: the state buffers hold 3*N*K*4 B = %.0f MB (L2 126 MB)"
              % (3 * (n + 1) ** 3 * a.K * 4 / 1e6),
    }


def problem(a):
    if a.mesh == "jitter":
        xyz, tets = S.jittered_cube_mesh(a.cells, 0.15, S.BATCHED.seed + 200)
    else:
        xyz, tets = S.cube_mesh(a.cells)
    if a.order != "native":
        from paper_2607_21373_b300 import reorder
        perm = (reorder.rcm_permutation(tets, xyz.shape[0]) if a.order == "rcm"
                else reorder.morton_permutation(xyz))
        xyz, tets = reorder.renumber(xyz, tets, perm)
    det = S.detector_points(a.n_obs, S.LIMITED_VIEW_FACES, S.BATCHED.seed)
    p0 = S.phantom(xyz, "blobs20+vessels", S.BATCHED.seed + 100, a.cells)
    return xyz, tets, det, p0, 0.3 / a.cells


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle timing (reported baseline and the reference arm)
# --------------------------------------------------------------------------
_W = {}


def _oracle_init(ops, p0, dt):
    _W.update(ops=ops, p0=p0, dt=dt)


def _oracle_solve(n_solve):
    """One oracle forward and one transposed solve of n_solve steps (K = 1);
    returns its wall time."""
    from oracle import wave
    t0 = time.perf_counter()
    Y = wave.forward(_W["ops"], _W["p0"], _W["dt"], n_solve)
    wave.adjoint(_W["ops"], Y, _W["dt"])
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The FP64 oracle (SciPy, single-threaded) in `procs` spawned processes,
    one RTO sample's wave solves per process (the paper's sample parallelism,
    Section 6.4).  Spawned, not forked, so the children hold no CUDA state."""

    def __init__(self, a, procs, problem_data=None):
        from oracle import fem
        xyz, tets, det, p0, dt = problem_data if problem_data else problem(a)
        ops = fem.build(xyz, tets, det, a.cells)
        self.N = len(xyz)
        self.procs = max(1, procs)
        lean = {k: ops[k] for k in ("K", "B", "ML", "Pi")}
        _oracle_init(lean, p0, dt)
        self.pool = None
        if self.procs > 1:
            for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
                os.environ[var] = "1"
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init, initargs=(lean, p0, dt))

    def rate(self, n_solve, reps=1):
        """Aggregate node-steps/s of `procs` concurrent forward + transposed
        solves of n_solve steps, repeated reps times; and the wall time."""
        t0 = time.perf_counter()
        for _ in range(reps):
            if self.pool is None:
                _oracle_solve(n_solve)
            else:
                self.pool.map(_oracle_solve, [n_solve] * self.procs, chunksize=1)
        sec = time.perf_counter() - t0
        return reps * self.procs * 2 * n_solve * self.N / sec, sec

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


def run_reference(a, rank, world):
    if rank != 0:
        return
    cfg = workload_config(a)
    nsps = cfg["node_steps_per_sample"]
    procs = a.cpu_procs or min(host_cores(), 64)
    pool = OraclePool(a, procs)
    n_solve = 50      # one step = one forward + one transposed solve of 50 time steps per process
    pool.rate(2)      # warm-up of every process (imports, first touch)
    for _ in range(a.warmup):
        pool.rate(n_solve)
    rate, sec = pool.rate(n_solve, reps=a.steps)
    pool.close()
    value = rate / nsps
    sample = (f"per step: {procs} oracle processes (one per host core), each one FP64 forward and one transposed "
              f"solve of {n_solve} of the {a.n_steps} time steps (K=1); samples/s extrapolated by node-steps: "
              f"{nsps:.3e} node-steps per sample")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * sec / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "node_steps_per_s": rate,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(a, data, nsps):
    """The oracle on the host cores: all cores (one process each), and one
    thread, on a bounded sample of the workload's wave solves."""
    procs = a.cpu_procs or min(host_cores(), 64)
    pool = OraclePool(a, procs, data)
    pool.rate(2)
    n_all = min(a.n_steps, 600)      # about 10 s of every core's time
    rate_all, sec_all = pool.rate(n_all)
    pool.close()
    one = OraclePool(a, 1, data)
    n_one = min(a.n_steps, 1000)
    rate_one, sec_one = one.rate(n_one)
    return {"value": rate_all / nsps, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} concurrent oracle processes (FP64 SciPy, one thread each), each one forward and one "
                      f"transposed solve of {n_all} of the {a.n_steps} steps on the same mesh (K=1), {sec_all:.1f} s; "
                      f"samples/s extrapolated by node-steps ({nsps:.3e} per sample)",
            "node_steps_per_s": rate_all,
            "one_thread": {"value": rate_one / nsps, "node_steps_per_s": rate_one,
                           "sample": f"one process, {n_one}-step forward + transposed solve, {sec_one:.1f} s"}}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def kernel_name(e, adj):
    """Readable name of the step-kernel variant an autotune entry describes."""
    tf = "true" if adj else "false"
    packed = e.get("packed")
    if packed == 7:
        return "step3u_persist_kernel<%s> (row pairs, %d blocks/SM)" % (tf, 3 if e.get("min_blocks") == 3 else 2)
    if packed == 8:
        return "step3q_persist_kernel<%s> (row quads%s)" % (tf, ", own rows async" if e.get("own_async") else "")
    if packed in (5, 6):
        if e.get("V") == 1:
            return "step3w1_kernel<%s> (16 slots, one sample%s)" % (tf, ", 6 blocks/SM" if e.get("min_blocks") == 6
                                                                     else "")
        nb = e.get("gather_batch") or 4
        big = bool(e.get("big_blocks"))
        return "step3w_persist_kernel<%s> (16 slots%s, rounds of %d%s%s%s)" % (
            tf, " row-major" if packed == 6 else "", nb,
            (", columns per round" if e.get("early") else "") + (
                ", 256-bit metadata" if packed == 6 and e.get("wide_loads") else ""),
            ", 1024-thread blocks" if big else (", 3 blocks/SM" if e.get("min_blocks") == 3 else ""),
            ", serial tail" if e.get("tail_serial") else "") + (" (own rows by bulk copy)" if e.get("own_async") == 2 else " (own x_{s-1} rows async)"
                                                    if e.get("own_async") == 3 else " (own rows async)" if e.get("own_async") else "") + (
            ((" (quad's coefficient lines to L1)" if packed == 5 else " (next metadata to L1)")
             if e.get("prefetch_meta") else "") + (" (chunks by counter)" if e.get("dyn_chunks") else ""))
    if packed == 2:
        return "step3t_kernel<8,%s>" % tf
    if packed == 4:
        return "step3p_kernel<%s> (persistent double-buffered tiles)" % tf
    if packed == 3:
        if e.get("V") == 1:
            return "step3e1_kernel<%s> (8 slots, one sample%s)" % (tf, ", 6 blocks/SM" if e.get("min_blocks") == 6
                                                                   else "")
        p = int(e.get("persistent") or 0)
        kind = {0: "step3e_kernel", 1: "step3e_persist_kernel", 2: "step3e_slab_kernel",
                3: "step3e_stage_kernel"}.get(p, "step3e_persistent(%d)" % p)
        flags = []
        if p:
            flags.append("1024-thread blocks" if e.get("big_blocks") else "256-thread blocks")
        if e.get("pdl"):
            flags.append("PDL")
        if e.get("prefetch"):
            flags.append("L2 prefetch %d" % e["prefetch"])
        if e.get("wide_loads"):
            flags.append("256-bit loads")
        if e.get("l2_hints"):
            flags.append("L2 hints")
        if e.get("gather_batch"):
            flags.append("batches of %d" % e["gather_batch"])
        if e.get("min_blocks", 1) > 1:
            flags.append(">=%d blocks/SM" % e["min_blocks"])
        return "%s<%d,%s>%s" % (kind, e.get("V", 0), tf, " (%s)" % ", ".join(flags) if flags else "")
    if packed:
        return "step3f_kernel<%d,%d,%s>%s" % (e.get("V", 0), e.get("chunk", 4), tf,
                                              " (Z-order rows)" if e.get("zorder") else "")
    return "step3_kernel<float,%d,split,%s,staged=%d>" % (e.get("V", 0), "adj" if adj else "fwd",
                                                          int(bool(e.get("staged"))))


def graph_operator_bytes(info, N):
    """Operator bytes per step on the full FEM graph as the scope table counts
    them: 4-byte column + 4-byte value per stiffness and boundary entry, row
    pointers and lumped mass of K (4 B each per node), row pointers of B."""
    return (info["nnz_K_graph"] * 8 + (N + 1) * 4 + N * 4 + info["nnz_B"] * 8
            + (info["n_boundary_nodes"] + 1) * 4)


def run_ours(a, rank, world, local_rank, dist):
    import torch

    from paper_2607_21373_b300 import Mesh
    from paper_2607_21373_b300.dist import allreduce_moments, first_sample

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = workload_config(a)
    data = problem(a)
    xyz, tets, det, p0, dt = data
    mesh = Mesh(xyz, tets, det, dt, a.n_steps, precision="f32", flags=mesh_flags(a))
    mesh.set_first_sample(first_sample(rank, a.K))   # rank r draws the global samples r*K .. r*K+K-1
    N = mesh.N
    # synthetic observations: Y = G p0 (our forward map), 1% relative noise (eq. noise-model)
    p0_d = torch.tensor(p0, dtype=torch.float32, device=dev)
    Y = mesh.forward(p0_d)
    gen = torch.Generator(device=dev)
    gen.manual_seed(S.BATCHED.seed + 2)
    eta0 = torch.randn(Y.shape, generator=gen, device=dev, dtype=torch.float32)
    sigma = float(S.BATCHED.noise * torch.linalg.vector_norm(Y.double()) / torch.linalg.vector_norm(eta0.double()))
    y_obs = (Y + sigma * eta0).contiguous()
    K, k = a.K, a.k_iter
    two_level = bool(mesh_flags(a) & MESH_TWO_LEVEL)
    # pick the step-kernel variant per direction for both sample counts (not timed)
    tune = {}
    names = a.variant.split(",") if a.variant else []
    forced = [FORCED[n] for n in names] if names else None
    if forced:
        forced = forced if len(forced) == 2 else forced * 2
        for d, v in zip(("fwd", "adj"), forced):
            mesh.select_variant(K, d, **v)
        tune["K%d" % K] = [dict(dict(direction=d, us_per_step=0.0), **v) for d, v in zip(("fwd", "adj"), forced)]
    elif a.autotune and not two_level:
        tune["K%d" % K] = mesh.autotune(K, n_probe=30)
    if a.autotune and not two_level and a.plain_steps > 0:
        tune["K1"] = mesh.autotune(1, n_probe=30)
    if a.tune_log and rank == 0:
        with open(a.tune_log, "w") as f:
            json.dump(tune, f)

    def batch(K_, seed):
        return mesh.rto_sample(y_obs, sigma, K_, k, seed=seed, samples=False, mean=True, stdev=K_ >= 2,
                               solver=a.solver)

    def barrier():
        if dist is not None:
            dist.barrier()

    for i in range(a.warmup):
        batch(K, i)
    mesh.status(K)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    mesh.profile_enable(True)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for i in range(a.steps):
        batch(K, 100 + i)
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = mesh.profile_read()
    mesh.profile_enable(False)
    clk = clocks.stop()
    mesh.status(K)
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        # pointwise posterior statistics over every rank's samples (outside the timed region)
        allreduce_moments(mesh, K)
    sec = ms / 1e3
    value = world * K * a.steps / sec
    nsps = cfg["node_steps_per_sample"]

    # roofline of the dominant kernel: the forward step (the transposed step beside it)
    info = mesh.info
    n_obs, NT = a.n_obs, a.n_steps
    # bytes per step as the scope table counts them: 16 B of state per node and
    # sample (read p, v; write p, v) + the full-graph operator; sensor I/O ignored
    alg_step = 16.0 * N * K + graph_operator_bytes(info, N)
    # bytes this library's step moves: 12 B of state (three-level form: read x_s,
    # x_{s-1}, write x_{s+1}; 16 B for the two-level form), its stored operator,
    # and the sensor reads / writes
    state_b = (16.0 if two_level else 12.0) * N * K
    fwd_moved = state_b + info["operator_bytes"] + n_obs * K * (3 * 8 + 4.0)
    adj_moved = state_b + info["operator_bytes"] + n_obs * 3 * 12.0 + 2 * n_obs * K * 4.0
    fwd_ms_launch = prof["fwd_ms"] / max(prof["fwd_launches"], 1)
    adj_ms_launch = prof["adj_ms"] / max(prof["adj_launches"], 1)
    per_launch = NT / (NT + 1.0)       # a forward solve: N_T steps + the final observation launch
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else None
    peak = peaks["hbm_gbs"] if peaks else 6400.0

    def gbs(b, ms_):
        return b * per_launch / (ms_ * 1e-3) / 1e9

    def best(direction):
        rows = [e for e in tune.get("K%d" % K, []) if e["direction"] == direction]
        return min(rows, key=lambda e: e["us_per_step"]) if rows else {}

    bf, ba = best("fwd"), best("adj")
    kname = "fwd_step_kernel<float,4,true>" if two_level else kernel_name(bf, False)
    aname = "adj_step_kernel<float,4,true>" if two_level else kernel_name(ba, True)
    default_shape = (a.cells, a.K, a.n_obs, a.mesh_flags) == (58, 64, 1024, 0)
    traffic = PROFILED_TRAFFIC.get((a.mesh, kname)) if default_shape else None
    ach = gbs(alg_step, fwd_ms_launch)
    roof = {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": traffic,
            "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6400 GB/s",
            "bytes_per_launch": alg_step * per_launch, "avg_launch_us": 1e3 * fwd_ms_launch,
            "bytes_rule": "16 B/node/sample of state + full-graph operator (nnz*8 + 8N + nnz_B*8 + 4N_b)",
            "moved": {"bytes_per_launch": fwd_moved * per_launch, "achieved": gbs(fwd_moved, fwd_ms_launch),
                      "frac": gbs(fwd_moved, fwd_ms_launch) / peak,
                      "rule": "12 B/node/sample (three-level state) + stored operator + sensor I/O"},
            "adjoint": {"kernel": aname, "avg_launch_us": 1e3 * adj_ms_launch,
                        "achieved": gbs(alg_step, adj_ms_launch), "frac": gbs(alg_step, adj_ms_launch) / peak,
                        "moved_frac": gbs(adj_moved, adj_ms_launch) / peak,
                        "traffic": PROFILED_TRAFFIC.get((a.mesh, aname)) if default_shape else None}}

    # plain one-sample form on the same library and workload
    plain = None
    if a.plain_steps > 0 and rank == 0:
        batch(1, 7)
        torch.cuda.synchronize()
        p0e, p1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0e.record(st)
        for i in range(a.plain_steps):
            batch(1, 9000 + i)
        p1e.record(st)
        torch.cuda.synchronize()
        psec = p0e.elapsed_time(p1e) / 1e3
        k1 = [e for e in tune.get("K1", []) if e["direction"] == "fwd"]
        plain = {"K": 1, "samples": a.plain_steps, "samples_per_s": a.plain_steps / psec,
                 "node_steps_per_s": a.plain_steps * nsps / psec, "ms_per_sample": 1e3 * psec / a.plain_steps,
                 "fwd_kernel": kernel_name(min(k1, key=lambda e: e["us_per_step"]), False) if k1 else None}

    # end to end through the public API with host buffers
    e2e = None
    if a.e2e_steps > 0:
        y_host = y_obs.cpu().pin_memory()
        mean_h = torch.empty(N, dtype=torch.float64).pin_memory()
        std_h = torch.empty(N, dtype=torch.float64).pin_memory()
        y_dev = torch.empty_like(y_obs)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(st)
        for i in range(a.e2e_steps):
            y_dev.copy_(y_host, non_blocking=True)
            out = mesh.rto_sample(y_dev, sigma, K, k, seed=5000 + i, samples=False, solver=a.solver)
            mean_h.copy_(out["mean"], non_blocking=True)
            std_h.copy_(out["std"], non_blocking=True)
        t1.record(st)
        torch.cuda.synchronize()
        esec = t0.elapsed_time(t1) / 1e3
        e2e = {"value": world * K * a.e2e_steps / esec, "unit": UNIT,
               "h2d_bytes_per_step": y_host.numel() * 4, "d2h_bytes_per_step": 2 * N * 8}

    cpu = None
    if rank == 0 and world == 1 and a.cpu_baseline:
        cpu = cpu_baseline(a, data, nsps)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "precision": "f32 state and stepping, f64 CGLS scalars, norms and iterate",
            "data": "synthetic (seeded mesh, phantom, noise, device draws)",
            "config": cfg, "node_steps_per_s": world * K * a.steps * nsps / sec,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": prof["total_launches"],
            "gpu_launches_per_step": prof["total_launches"] / a.steps, "clocks": clk, "plain": plain,
            "batched_over_plain": (value / world) / plain["samples_per_s"] if plain else None,
            "variants": {"fwd": kname, "adj": aname,
                         "fwd_us": bf.get("us_per_step"), "adj_us": ba.get("us_per_step"),
                         "timed": sum(len(v) for v in tune.values())},
        }
        print(json.dumps(line), flush=True)


def run_uneven(a, rank, world, local_rank, dist):
    """Uneven batch: the six jobs of S.UNEVEN (cubes of 16^3..58^3 cells, N_T =
    1000 n / 58, sensors 1024 (n / 58)^2 on five faces, K = 256..8, noise 1-4 %,
    CGLS k = 50) in one grouped solve (pat_rto_sample_multi) per step."""
    import torch

    from paper_2607_21373_b300 import Mesh, rto_sample_multi

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    jobs, info = [], []
    for w in S.UNEVEN:
        xyz, tets = S.cube_mesh(w.n)
        det = S.detector_points(w.n_obs, w.faces, w.seed)
        p0 = S.phantom(xyz, w.phantom, w.seed + 100, w.n)
        m = Mesh(xyz, tets, det, w.dt_factor / w.n, w.n_steps, precision="f32", flags=mesh_flags(a))
        m.set_first_sample(rank * w.K)
        Y = m.forward(torch.tensor(p0, dtype=torch.float32, device=dev))
        gen = torch.Generator(device=dev)
        gen.manual_seed(w.seed + 2)
        eta0 = torch.randn(Y.shape, generator=gen, device=dev, dtype=torch.float32)
        sigma = float(w.noise * torch.linalg.vector_norm(Y.double()) / torch.linalg.vector_norm(eta0.double()))
        jobs.append({"mesh": m, "y_obs": (Y + sigma * eta0).contiguous(), "sigma": sigma, "K": w.K, "seed": w.seed})
        info.append({"n": w.n, "N": m.N, "N_T": w.n_steps, "n_obs": w.n_obs, "K": w.K, "noise": w.noise,
                     "op_bytes": graph_operator_bytes(m.info, m.N)})
    k = S.UNEVEN[0].n_iter
    for i in range(a.warmup):
        rto_sample_multi(jobs, k, samples=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    e0.record(st)
    for i in range(a.steps):
        rto_sample_multi(jobs, k, samples=False)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    for j in jobs:
        j["mesh"].status(j["K"])
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    sec = ms / 1e3
    ksum = sum(w["K"] for w in info)
    node_steps = sum((2 * k + 1) * w["N_T"] * w["N"] * w["K"] for w in info)
    alg_bytes = sum((2 * k + 1) * w["N_T"] * (16.0 * w["N"] * w["K"] + w["op_bytes"]) for w in info)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = json.load(open(peaks_path))["hbm_gbs"] if os.path.exists(peaks_path) else 6400.0
    if rank == 0:
        line = {
            "metric": METRIC, "value": world * ksum * a.steps / sec, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded meshes, phantoms, noise, device draws)",
            "config": {"workload": "uneven batch: six cubes %s^3 cells, K %s, one grouped CGLS k=%d solve per step, "
                                   "mesh %s" % ("/".join(str(w["n"]) for w in info),
                                                "/".join(str(w["K"]) for w in info), k, a.mesh),
                       "jobs": [{kk: w[kk] for kk in ("n", "N", "N_T", "n_obs", "K", "noise")} for w in info]},
            "node_steps_per_s": world * node_steps * a.steps / sec,
            "per_job_samples_per_s": [w["K"] * a.steps / sec for w in info],
            "roofline": {"bound": "hbm", "kernel": "step3g_persist_kernel (grouped fixed-width steps)",
                         "achieved": alg_bytes * a.steps / sec / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg_bytes * a.steps / sec / 1e9 / peak, "traffic": None,
                         "note": "whole-step average (vector kernels and launch gaps included): a lower bound "
                                 "on the step kernels' own rate"},
            "cpu_baseline": None, "e2e": None, "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def run_matern(a, rank, world, local_rank, dist):
    """The rto workload's mesh, sensors and data with the Whittle-Matern prior of
    Section 6.4 (l = 0.15, s = 1.5, sigma = 3, 128^3 grid on a periodic box
    holding the cube with 0.5 to spare on every side): K latent-space RTO
    samples (CGLS, k iterations) per step."""
    import torch

    from paper_2607_21373_b300 import MaternPrior, Mesh

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    xyz, tets, det, p0, dt = problem(a)
    mesh = Mesh(xyz, tets, det, dt, a.n_steps, precision="f32", flags=mesh_flags(a))
    mesh.set_first_sample(rank * a.K)
    ng = 128
    prior = MaternPrior(mesh, ng, (-0.5, -0.5, -0.5), 2.0, 0.15, 1.5, 3.0)
    Y = mesh.forward(torch.tensor(p0, dtype=torch.float32, device=dev))
    gen = torch.Generator(device=dev)
    gen.manual_seed(S.BATCHED.seed + 2)
    eta0 = torch.randn(Y.shape, generator=gen, device=dev, dtype=torch.float32)
    sigma = float(S.BATCHED.noise * torch.linalg.vector_norm(Y.double()) / torch.linalg.vector_norm(eta0.double()))
    y_obs = (Y + sigma * eta0).contiguous()
    K, k = a.K, a.k_iter
    if a.autotune:
        mesh.autotune(K, n_probe=30)
    for i in range(a.warmup):
        prior.rto_sample(y_obs, sigma, K, k, seed=i, samples=False)
    prior.status(K)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    mesh.profile_enable(True)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in range(a.steps):
        prior.rto_sample(y_obs, sigma, K, k, seed=100 + i, samples=False)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = mesh.profile_read()
    mesh.profile_enable(False)
    clk = clocks.stop()
    prior.status(K)
    sec = ms / 1e3
    wave_ms = prof["fwd_ms"] + prof["adj_ms"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": world * K * a.steps / sec, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded mesh, phantom, noise, device draws)",
            "config": dict(workload_config(a), prior="Whittle-Matern: 128^3 periodic grid on [-0.5, 1.5)^3, l=0.15, "
                                                     "s=1.5, sigma=3; RTO in the latent space (CGLS k=%d)" % k),
            "wave_solve_share": wave_ms / ms, "cpu_baseline": None, "e2e": None, "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def run_grad(a, rank, world, local_rank, dist):
    """Differentiation workload: 32^3-cell cube (35,937 nodes), 1000 steps, 256
    sensors on five faces, per-element c = sqrt(c2) from a smoothed N(0, 1)
    field (amplitude 0.1), FP32 state on the full P1 graph.  One step = one
    gradient evaluation of L = 1/2 ||G(c2) p0 - y||^2 for K stacked p0
    (pat_grad_c2: dL/dc2 summed over the samples and dL/dp0, the forward
    trajectory recomputed from ceil(sqrt(N_T)) checkpoints)."""
    import torch

    from paper_2607_21373_b300 import Mesh

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = S.DIFFERENTIATION
    n = a.cells if a.cells_given else w.n
    nt = a.n_steps if a.n_steps_given else w.n_steps
    n_obs = a.n_obs if a.n_obs_given else w.n_obs
    K = a.K if a.K_given else w.K
    xyz, tets = S.cube_mesh(n)
    det = S.detector_points(n_obs, w.faces, w.seed)
    c2 = S.smoothed_speed_field(n, w.seed + 7)
    dt = w.dt_factor / n / float(np.sqrt(c2.max()))
    mesh = Mesh(xyz, tets, det, dt, nt, precision="f32", c2=c2, flags=MESH_KEEP_ZEROS)
    N, E = mesh.N, mesh.info["n_tets"]
    p0 = S.phantom(xyz, w.phantom, w.seed + 100, n)
    P = np.stack([p0 * (1.0 + 0.05 * k) for k in range(K)], axis=1) if K > 1 else p0
    p_d = torch.tensor(P, dtype=torch.float32, device=dev)
    # data from a 10 % weaker initial pressure, so the misfit cotangent is not zero
    y = mesh.forward(0.9 * p_d)
    tune = []
    if a.variant:
        forced = [FORCED[v] for v in a.variant.split(",")]
        forced = forced if len(forced) == 2 else forced * 2
        for d, v in zip(("fwd", "adj"), forced):
            mesh.select_variant(K, d, **v)
        tune = [dict(dict(direction=d, us_per_step=0.0), **v) for d, v in zip(("fwd", "adj"), forced)]
    elif a.autotune:
        tune = mesh.autotune(K, n_probe=30)
    if a.tune_log and rank == 0:
        with open(a.tune_log, "w") as f:
            json.dump({"K%d" % K: tune}, f)

    def best(direction):
        rows = [e for e in tune if e["direction"] == direction]
        return min(rows, key=lambda e: e["us_per_step"]) if rows else None

    yhat = (mesh.forward(p_d) - y).contiguous()
    g = torch.empty(E, dtype=torch.float64, device=dev)
    pg = torch.empty_like(p_d)
    for i in range(a.warmup):
        mesh.grad_c2(p_d, yhat, out=(g, pg))
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    e0.record(st)
    for i in range(a.steps):
        mesh.grad_c2(p_d, yhat, out=(g, pg))
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    if not (torch.isfinite(g).all() and torch.isfinite(pg).all()):
        raise RuntimeError("non-finite gradient")
    # end to end: p0 and the cotangent from pinned host memory, both gradients back
    p_h, y_h = p_d.cpu().pin_memory(), yhat.cpu().pin_memory()
    g_h = torch.empty(E, dtype=torch.float64).pin_memory()
    pg_h = torch.empty(pg.shape, dtype=torch.float32).pin_memory()
    p_in, y_in = torch.empty_like(p_d), torch.empty_like(yhat)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in range(a.steps):
        p_in.copy_(p_h, non_blocking=True)
        y_in.copy_(y_h, non_blocking=True)
        mesh.grad_c2(p_in, y_in, out=(g, pg))
        g_h.copy_(g, non_blocking=True)
        pg_h.copy_(pg, non_blocking=True)
    e2.record(st)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e2)
    if dist is not None:
        t = torch.tensor([ms, ms_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_e2e = float(t[0]), float(t[1])
    L = int(np.ceil(np.sqrt(nt)))
    n_ck = (nt + L - 1) // L
    launches = (nt - 1) + (nt - n_ck) + (nt + 1)  # forward sweep, recomputation, transposed sweep
    node_steps = launches * N * K
    op_bytes = graph_operator_bytes(mesh.info, N)
    elem_bytes = n_ck * E * (16 + 40 + 16) + nt * E * 8 * K * 1.0  # tets, coefficients, g; 8 state values a step
    alg_bytes = launches * (16.0 * N * K + op_bytes) + elem_bytes
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = json.load(open(peaks_path))["hbm_gbs"] if os.path.exists(peaks_path) else 6400.0
    sec = ms / 1e3
    cpu = None
    if rank == 0 and a.cpu_baseline:
        from oracle import fem, gradient
        steps_cpu = min(nt, 200)
        ops = gradient.with_c2(fem.build(xyz, tets, det, n), tets, c2)
        y_cpu = (y[:steps_cpu, :, 0] if K > 1 else y[:steps_cpu]).double().cpu().numpy()
        t0 = time.perf_counter()
        gradient.gradients(ops, tets, p0, y_cpu, dt)
        t_cpu = (time.perf_counter() - t0) * nt / steps_cpu
        cpu = {"value": 1.0 / (t_cpu * K), "unit": "gradients/s", "cores": 1, "kind": "oracle",
               "sample": "one FP64 oracle gradient (forward and reverse sweep, all states kept) over %d of the %d "
                         "steps, one sample, %.1f s; extrapolated by steps" % (steps_cpu, nt, t_cpu * steps_cpu / nt)}
    if rank == 0:
        line = {
            "metric": "grad_c2_evaluations_per_s", "value": world * a.steps / sec, "unit": "gradients/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded mesh, sound-speed field, phantom)",
            "config": {"workload": "cube%d_grad: unit cube %d^3 cells x 6 tets (full P1 graph), %d nodes, N_T=%d, "
                                   "%d sensors on 5 faces, c = sqrt(c2) smoothed field (amplitude 0.1), K=%d "
                                   "stacked misfits, %d checkpoints" % (n, n, N, nt, n_obs, K, n_ck),
                       "n_nodes": N, "n_tets": E, "n_steps": nt, "K": K, "checkpoints": n_ck,
                       "l2": "state and operator (%.0f MB) stay in L2" % ((4 * N * K * 4 + op_bytes) / 1e6)},
            "node_steps_per_s": world * node_steps * a.steps / sec,
            "roofline": {"bound": "hbm", "kernel": "whole evaluation (step kernels and segment element passes)",
                         "achieved": alg_bytes * a.steps / sec / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg_bytes * a.steps / sec / 1e9 / peak, "traffic": None,
                         "note": "scope bytes of every step launch plus the element passes over the whole "
                                 "evaluation; the working set stays in L2, so the launches are latency-bound"},
            "cpu_baseline": cpu,
            "e2e": {"value": world * a.steps / (ms_e2e / 1e3), "unit": "gradients/s",
                    "h2d_bytes_per_step": int(p_h.numel() * 4 + y_h.numel() * 4),
                    "d2h_bytes_per_step": int(E * 8 + pg_h.numel() * 4)},
            "gpu_launches": a.steps * (launches + n_ck + 1), "clocks": clk,
            "variants": {d: ({"kernel": kernel_name(b, d == "adj"), "us_per_step": b["us_per_step"]}
                             if b else "library default") for d, b in (("fwd", best("fwd")), ("adj", best("adj")))},
        }
        print(json.dumps(line), flush=True)


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        backend = "nccl" if (a.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        tdist.init_process_group(backend)
        dist = tdist
    if a.impl == "reference":
        run_reference(a, rank, world)
    elif a.workload == "uneven":
        run_uneven(a, rank, world, local_rank, dist)
    elif a.workload == "matern":
        run_matern(a, rank, world, local_rank, dist)
    elif a.workload == "grad":
        run_grad(a, rank, world, local_rank, dist)
    else:
        run_ours(a, rank, world, local_rank, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
