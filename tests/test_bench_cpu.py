"""Host logic of bench.py that runs after the timed region: naming every step-kernel
variant the autotuner can report (a missing case would lose the whole bench line)."""
import itertools
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_every_autotune_entry_has_a_kernel_name():
    seen = set()
    for packed, persist, big, pdl, pf, wide, hint, gb, mb, V in itertools.product(
            range(5), range(4), (0, 1), (0, 1), (0, 1, 2), (0, 1), (0, 1), (0, 2, 4, 8), (1, 5, 6), (1, 2, 4, 8)):
        e = dict(direction="fwd", V=V, staged=False, packed=packed, chunk=4, min_blocks=mb, early=False,
                 zorder=False, big_blocks=bool(big), prefetch=pf, persistent=persist, pdl=bool(pdl),
                 wide_loads=bool(wide), l2_hints=bool(hint), gather_batch=gb, us_per_step=1.0)
        for adj in (False, True):
            seen.add(bench.kernel_name(e, adj))
    assert "step3e_stage_kernel<8,false> (256-thread blocks, PDL)" in seen
    assert "step3e_persist_kernel<8,true> (1024-thread blocks, PDL)" in seen
    assert set(bench.PROFILED_TRAFFIC) <= seen


def test_workload_config_names_the_solver():
    class A:
        cells, n_steps, n_obs, K, k_iter, solver = 58, 1000, 1024, 64, 100, "lsqr"
    c = bench.workload_config(A)
    assert c["solver"] == "lsqr" and c["lsqr_iters"] == 100 and c["n_nodes"] == 59 ** 3
