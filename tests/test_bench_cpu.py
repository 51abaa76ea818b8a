"""Host-side arithmetic of the benchmark line that needs no GPU: the assembly-only rate
(design rows over the device time of the kernel classes gap_assemble runs)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_assembly_rate_sums_the_assembly_classes_only():
    b = load_bench()
    # per-step kernel-class times of a workload-2 step (441,968 data rows), in ms
    phases = {"pack": 9.327, "gemm_energy": 9.275, "gemm_force": 112.38, "kmm_chol": 14.465,
              "qr_update": 95.552, "solve": 1.642, "refine": 28.841, "predict": 14.516, "copy_in": 0.0}
    a = b.assembly_rate(phases, 441968)
    assert a["ms"] == pytest.approx(9.327 + 9.275 + 112.38)
    assert a["rows_per_s"] == pytest.approx(441968 / 0.130982)
    assert a["phases"] == ["pack", "gemm_energy", "gemm_force"]
    # a host problem's staging counts as assembly
    a5 = b.assembly_rate({"copy_in": 577.1, "pack": 41.3, "gemm_energy": 89.3, "gemm_force": 2150.2,
                          "qr_update": 2192.0}, 1011291)
    assert a5["ms"] == pytest.approx(577.1 + 41.3 + 89.3 + 2150.2)
    assert a5["phases"][0] == "copy_in"
    assert b.assembly_rate({}, 10)["rows_per_s"] is None


def test_launch_count_matches_the_committed_launch_list():
    """kernel_launch_count, the line's gpu_launches, against the ncu launch list of the
    workload-2 mixed_bf16 step (M = 4000, d = 512) committed with the profiles: 2052 kernel
    launches per step at 13 refinement iterations, and 16 launches per iteration."""
    import types
    b = load_bench()
    p = types.SimpleNamespace(n_sparse=4000, d=512)
    assert b.kernel_launch_count(p, "mixed_bf16", 13) == 2052
    assert b.kernel_launch_count(p, "mixed_bf16", 12) == 2036  # the slice run's 4072 launches over 2 steps
    assert b.kernel_launch_count(p, "mixed_bf16", 11) == 2020
