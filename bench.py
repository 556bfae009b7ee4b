#!/usr/bin/env python
"""Throughput of the batched RTO sampler on B300 (one JSON line on stdout).

One step = one RTO batch: K posterior samples, each the CGLS solve of the
extended least-squares system with k iterations (2k+1 wave solves of N_T steps
per sample), on a seeded synthetic workload shaped like the paper's 3D problem
(Section 6.4: ~2e5 unknowns): unit cube 58^3 cells x 6 tets (205,379 nodes),
N_T = 1000, 1024 sensors on five faces, K = 64, k = 100, FP32 state with FP64
CGLS scalars.  The timed region holds the whole batch (data perturbations and
prior draws come from the library's counter-based generator on the device).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own K samples (sample parallelism, no data
collective; weak scaling); rank 0 prints the line.  --impl reference times the
FP64 CPU oracle on the same workload (a bounded, extrapolated sample).
"""
from __future__ import annotations

import argparse
import json
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
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one step launch, from
# one ncu capture of that kernel variant on the default workload (cube58, K = 64,
# 1024 sensors); see profiles/step3e_persist_kernel_cube58_K64.md.  Used for the
# roofline's "traffic" only when the timed run uses the same variant and workload.
PROFILED_TRAFFIC = {
    "step3e_persist_kernel<8,false> (256-thread blocks, PDL, L2 prefetch 1)": 160.643584e6,
    "step3e_persist_kernel<8,true> (256-thread blocks, PDL, L2 prefetch 1)": 159.604480e6,
    "step3e_persist_kernel<8,false> (1024-thread blocks, PDL)": 159.210752e6,
    "step3e_persist_kernel<8,true> (1024-thread blocks, PDL)": 158.733312e6,
}
UNIT = "samples/s"


def parse():
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
    ap.add_argument("--plain-steps", type=int, default=1, help="timed K=1 batches (0: skip the plain form)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--mesh-flags", type=int, default=0, help="pat_mesh_create flags (e.g. 16: two-level form)")
    ap.add_argument("--autotune", type=int, default=1, help="0: keep the library's default step-kernel variant")
    ap.add_argument("--solver", default="cgls", choices=["cgls", "lsqr"],
                    help="least-squares solver of every RTO sample (the configured workload names CGLS)")
    ap.add_argument("--variant", default="", help="force a step-kernel variant for K: tiled | v8c2 | v4c4 | v8c2z | ell8 | ell4 | pipe | "
                    "ell8pf | ell8p | ell8pw | ell8pp | ell8pb")
    return ap.parse_args()


def workload_config(a):
    w = S.BATCHED
    return {
        "workload": f"cube{a.cells}_rto: unit cube {a.cells}^3 cells x 6 Kuhn tets, {(a.cells + 1) ** 3} nodes, "
                    f"N_T={a.n_steps}, dt=0.3h, {a.n_obs} sensors on 5 faces, K={a.K} samples per batch, "
                    f"{a.solver.upper()} k={a.k_iter}, white-noise prior N(0, M_L^-1), 1% noise",
        "n_nodes": (a.cells + 1) ** 3, "n_tets": 6 * a.cells ** 3, "n_steps": a.n_steps, "n_obs": a.n_obs,
        "K": a.K, "solver": a.solver, "cgls_iters" if a.solver == "cgls" else "lsqr_iters": a.k_iter,
        "noise": w.noise,
        "node_steps_per_sample": (2 * a.k_iter + 1) * a.n_steps * (a.cells + 1) ** 3,
        "l2": "inputs larger than L2: the K-stacked state is 4*N*K*4 B = %.0f MB per buffer set"
              % (4 * (a.cells + 1) ** 3 * a.K * 4 / 1e6),
    }


def problem(a):
    xyz, tets = S.cube_mesh(a.cells)
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
def oracle_rate(a, n_solve_steps, xyz=None, tets=None, det=None, p0=None):
    """Oracle node-steps/s over one forward and one transposed solve of
    n_solve_steps steps each (K = 1), single-threaded SciPy."""
    from oracle import fem, wave
    if xyz is None:
        xyz, tets, det, p0, _ = problem(a)
    dt = 0.3 / a.cells
    ops = fem.build(xyz, tets, det, a.cells)
    t0 = time.perf_counter()
    Y = wave.forward(ops, p0, dt, n_solve_steps)
    wave.adjoint(ops, Y, dt)
    sec = time.perf_counter() - t0
    return 2 * n_solve_steps * len(xyz) / sec, sec


def run_reference(a, rank, world):
    if rank != 0:
        return
    cfg = workload_config(a)
    nsps = cfg["node_steps_per_sample"]
    xyz, tets, det, p0, _ = problem(a)
    from oracle import fem, wave
    ops = fem.build(xyz, tets, det, a.cells)
    dt = 0.3 / a.cells
    n_solve = 50      # one step = one forward + one transposed solve of 50 time steps

    def one():
        Y = wave.forward(ops, p0, dt, n_solve)
        wave.adjoint(ops, Y, dt)

    for _ in range(a.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        one()
    sec = time.perf_counter() - t0
    node_steps = a.steps * 2 * n_solve * len(xyz)
    value = node_steps / sec / nsps
    sample = (f"per step: one FP64 oracle forward and one transposed solve of {n_solve} of the {a.n_steps} time "
              f"steps (K=1); samples/s extrapolated by node-steps: {nsps:.3e} node-steps per sample")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * sec / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "node_steps_per_s": node_steps / sec,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def kernel_name(e, adj):
    """Readable name of the step-kernel variant an autotune entry describes."""
    tf = "true" if adj else "false"
    packed = e.get("packed")
    if packed == 2:
        return "step3t_kernel<8,%s>" % tf
    if packed == 4:
        return "step3p_kernel<%s> (persistent double-buffered tiles)" % tf
    if packed == 3:
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


def run_ours(a, rank, world, local_rank, dist):
    import torch

    from paper_2607_21373_b300 import Mesh

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = workload_config(a)
    xyz, tets, det, p0, dt = problem(a)
    mesh = Mesh(xyz, tets, det, dt, a.n_steps, precision="f32", flags=a.mesh_flags)
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
    # pick the step-kernel variant per direction for both sample counts (not timed)
    tune = {}
    forced = {"tiled": dict(V=8, packed=2), "v8c2": dict(V=8, packed=1, chunk=2),
              "v4c4": dict(V=4, packed=1, chunk=4), "v8c2z": dict(V=8, packed=1, chunk=2, zorder=True),
              "ell8": dict(V=8, packed=3), "ell4": dict(V=4, packed=3), "pipe": dict(V=8, packed=4),
              "ell8pf": dict(V=8, packed=3, prefetch=1),
              "ell8p": dict(V=8, packed=3, persistent=True),
              "ell8pw": dict(V=8, packed=3, persistent=True, pdl=True, wide_loads=True, prefetch=1),
              "ell8pp": dict(V=8, packed=3, persistent=1, pdl=True, prefetch=1),
              "ell8pb": dict(V=8, packed=3, persistent=1, pdl=True, big_blocks=True)}.get(a.variant)
    if forced:
        for d in ("fwd", "adj"):
            mesh.select_variant(K, d, **forced)
        tune["K%d" % K] = [dict(dict(direction=d, us_per_step=0.0, staged=False, chunk=0), **forced)
                           for d in ("fwd", "adj")]
    elif a.autotune and not (a.mesh_flags & 0x10):
        tune["K%d" % K] = mesh.autotune(K, n_probe=30)
        if a.plain_steps > 0:
            tune["K1"] = mesh.autotune(1, n_probe=30)

    def batch(K_, seed):
        return mesh.rto_sample(y_obs, sigma, K_, k, seed=seed, samples=False, mean=True, stdev=K_ >= 2,
                               solver=a.solver)

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2607_21373_b300.dist import allreduce_moments, sample_seed
    for i in range(a.warmup):
        batch(K, sample_seed(i, rank))
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
        last = batch(K, sample_seed(100 + i, rank))
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
        allreduce_moments(last["mean"], last["std"], K)
    sec = ms / 1e3
    value = world * K * a.steps / sec
    nsps = cfg["node_steps_per_sample"]

    # roofline of the dominant kernel (forward step; the transposed step is reported beside it)
    info = mesh.info
    n_obs, NT = a.n_obs, a.n_steps
    two_level = bool(a.mesh_flags & 0x10)
    # per node and sample: two-level reads a, w and writes a, w (16 B); three-level reads
    # x_s, x_{s-1} and writes x_{s+1} (12 B)
    state_b = (16.0 if two_level else 12.0) * N * K
    gather_b = n_obs * K * (3 * 8 + 4.0)         # sensor reads of two fields at 3 nodes + the observation write
    fwd_loop_bytes = NT * (state_b + info["operator_bytes"]) + NT * gather_b
    fwd_launch_per_loop = NT + 1
    fwd_avg_ms = prof["fwd_ms"] / max(prof["fwd_launches"], 1)
    fwd_bytes_per_launch = fwd_loop_bytes / fwd_launch_per_loop
    if two_level:
        adj_op_b = info["operator_bytes"] + 8.0 * N + n_obs * 3 * 12.0
        adj_loop_bytes = NT * (state_b + adj_op_b) + NT * n_obs * K * 4.0
    else:
        adj_op_b = info["operator_bytes"] + n_obs * 3 * 12.0
        adj_loop_bytes = NT * (state_b + adj_op_b) + NT * 2 * n_obs * K * 4.0
    adj_avg_ms = prof["adj_ms"] / max(prof["adj_launches"], 1)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    achieved = fwd_bytes_per_launch / (fwd_avg_ms * 1e-3) / 1e9
    adj_achieved = (adj_loop_bytes / (NT + 1)) / (adj_avg_ms * 1e-3) / 1e9
    def best(direction):
        rows = [e for e in tune.get("K%d" % K, []) if e["direction"] == direction]
        return min(rows, key=lambda e: e["us_per_step"]) if rows else {"V": 4, "staged": False, "packed": True}

    bf, ba = best("fwd"), best("adj")
    default_workload = (a.cells, a.K, a.n_obs, a.mesh_flags) == (58, 64, 1024, 0)
    kname = "fwd_step_kernel<float,4,true>" if two_level else kernel_name(bf, False)
    aname = "adj_step_kernel<float,4,true>" if two_level else kernel_name(ba, True)
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak,
            "traffic": PROFILED_TRAFFIC.get(kname) if default_workload else None,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback",
            "bytes_per_launch": fwd_bytes_per_launch, "avg_launch_us": 1e3 * fwd_avg_ms,
            "traffic_source": "ncu capture of the same variant, profiles/step3e_persist_kernel_cube58_K64.md",
            "adjoint": {"kernel": aname, "achieved": adj_achieved,
                        "frac": adj_achieved / peak, "avg_launch_us": 1e3 * adj_avg_ms,
                        "traffic": PROFILED_TRAFFIC.get(aname) if default_workload else None}}

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
        plain = {"K": 1, "samples_per_s": a.plain_steps / psec, "node_steps_per_s": a.plain_steps * nsps / psec,
                 "ms_per_sample": 1e3 * psec / a.plain_steps}

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
        n_solve = a.n_steps
        rate, csec = oracle_rate(a, n_solve, xyz, tets, det, p0)
        cpu = {"value": rate / nsps, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one FP64 oracle forward and one transposed solve of {n_solve} steps on the same mesh "
                         f"(K=1, single-threaded SciPy, {csec:.1f} s); samples/s extrapolated by node-steps "
                         f"({nsps:.3e} per sample)", "node_steps_per_s": rate}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 state, f64 CGLS scalars", "data": "synthetic (seeded cube mesh, phantom, noise, draws)",
            "config": cfg, "node_steps_per_s": world * K * a.steps * nsps / sec,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": prof["total_launches"],
            "gpu_launches_per_step": prof["total_launches"] / a.steps, "clocks": clk, "plain": plain,
            "batched_over_plain": (value / world) / plain["samples_per_s"] if plain else None,
            "autotune": tune,
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
    else:
        run_ours(a, rank, world, local_rank, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
