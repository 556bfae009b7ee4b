"""Host logic of bench.py: naming every step-kernel variant the autotuner can
report (a missing case would lose the whole bench line), the workload record,
and the reference arm (the FP64 oracle in spawned processes) end to end on a
small cube."""
import itertools
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_every_autotune_entry_has_a_kernel_name():
    seen = set()
    for packed, persist, big, pdl, pf, wide, hint, gb, mb, V, early, tail, own in itertools.product(
            range(8), range(4), (0, 1), (0, 1), (0, 1, 2), (0, 1), (0, 1), (0, 2, 4, 8), (1, 3, 5, 6), (1, 2, 4, 8),
            (0, 1), (0, 1), (0, 1)):
        e = dict(direction="fwd", V=V, staged=False, packed=packed, chunk=4, min_blocks=mb, early=bool(early),
                 zorder=False, big_blocks=bool(big), prefetch=pf, persistent=persist, pdl=bool(pdl),
                 wide_loads=bool(wide), l2_hints=bool(hint), gather_batch=gb, tail_serial=bool(tail),
                 own_async=bool(own), us_per_step=1.0)
        for adj in (False, True):
            seen.add(bench.kernel_name(e, adj))
    for packed, own, pfm, dyn, early, tail in itertools.product((5, 6, 7, 8), (0, 1, 2, 3), (0, 1), (0, 1), (0, 1),
                                                                (0, 1)):
        e = dict(direction="adj", V=8, packed=packed, gather_batch=4, early=bool(early), tail_serial=bool(tail),
                 own_async=own, prefetch_meta=bool(pfm), dyn_chunks=bool(dyn), us_per_step=1.0)
        for adj in (False, True):
            seen.add(bench.kernel_name(e, adj))
    assert "step3e_stage_kernel<8,false> (256-thread blocks, PDL)" in seen
    assert "step3e_persist_kernel<8,true> (1024-thread blocks, PDL)" in seen
    assert "step3w_persist_kernel<false> (16 slots, rounds of 8, columns per round)" in seen
    assert {name for _, name in bench.PROFILED_TRAFFIC} <= seen


def test_workload_config_names_the_solver_and_mesh():
    a = bench.parse(["--solver", "lsqr", "--mesh", "jitter"])
    c = bench.workload_config(a)
    assert c["solver"] == "lsqr" and c["iters"] == 100 and c["n_nodes"] == 59 ** 3 and c["mesh"] == "jitter"
    assert bench.mesh_flags(a) & bench.MESH_KEEP_ZEROS
    assert not bench.mesh_flags(bench.parse(["--mesh", "pruned"])) & bench.MESH_KEEP_ZEROS


def test_gradient_workload_takes_the_differentiation_sizes_unless_given():
    a = bench.parse(["--workload", "grad"])
    assert a.workload == "grad" and not (a.cells_given or a.n_steps_given or a.n_obs_given or a.K_given)
    b = bench.parse(["--workload", "grad", "--K", "8", "--cells=16"])
    assert b.K_given and b.cells_given and b.K == 8 and b.cells == 16 and not b.n_steps_given
    w = bench.S.DIFFERENTIATION
    assert (w.n, w.n_steps, w.n_obs, w.K) == (32, 1000, 256, 1)
    assert bench.kernel_name(bench.FORCED["e1"], False) == "step3e1_kernel<false> (8 slots, one sample)"


def test_reference_arm_prints_one_parsable_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--cells", "6", "--n-steps", "60",
           "--n-obs", "16", "--steps", "2", "--warmup", "1", "--cpu-procs", "2"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1 and len(lines[0]) < 4096
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["cpu_baseline"]["cores"] == 2
    assert rec["e2e"]["h2d_bytes_per_step"] == 0
