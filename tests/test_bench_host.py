"""Host-side arithmetic of the bench's roofline objects (no GPU): the
branch-weighted FP32 march flops, the FP32 replay's bandwidth figure, and
the small profiling workload."""

import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_fp32_march_roofline_weights_the_counted_branch_mix():
    m32 = {"ms_per_launch": 10.0, "steps_per_launch": 1_000_000_000,
           "branch_count_steps": 1_000_000_000, "series_steps": 750_000_000}
    r = bench.fp32_roofline(m32, {"fp32_tflops": 80.0})
    flops = 0.75 * bench.FLOPS_SERIES_FP32 + 0.25 * bench.FLOPS_CLOSED_FP32
    assert r["flops_per_step"] == pytest.approx(flops, abs=0.01)
    assert r["achieved"] == pytest.approx(flops * 1e9 / 1e-2 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.PEAK_FP32_TFLOPS, rel=1e-3)
    assert r["achieved_closed_form_only"] < r["achieved"]
    assert r["issue"]["frac"] == pytest.approx(
        bench.INSTR_PER_STEP_FP32 * 1e9 / 1e-2 / 1e12 / bench.PEAK_ISSUE_TINST, rel=1e-3)
    # without a branch count the closed-form count is the figure
    r0 = bench.fp32_roofline({"ms_per_launch": 10.0, "steps_per_launch": 1_000_000_000}, {"fp32_tflops": None})
    assert r0["flops_per_step"] == bench.FLOPS_PER_STEP_FP32
    assert r0["series_fraction"] is None


def test_fp32_replay_roofline_is_its_dram_bytes_over_time():
    r = bench.fp32_replay_roofline({"ms_per_launch": 5.0, "steps_per_launch": 3_000_000_000})
    gbs = bench.REPLAY32_DRAM_BYTES_PER_STEP * 3e9 / 5e-3 / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(gbs, rel=1e-3)
    assert r["frac"] == pytest.approx(gbs / bench.MEASURED_HBM_GBS, rel=1e-3)
    assert r["achieved_tflops"] == pytest.approx(
        bench.FLOPS_PER_STEP_FP32_REPLAY * 3e9 / 5e-3 / 1e12, rel=1e-3)


def test_branch_flop_counts_are_consistent():
    # both branches share the common part; the series branch does more
    assert bench.FLOPS_SERIES_FP32 > bench.FLOPS_CLOSED_FP32 > bench.FLOPS_COMMON_FP32
    assert bench.FLOPS_PER_STEP_FP32 == bench.FLOPS_CLOSED_FP32


def test_small_profiling_workload():
    p = bench.make_problem("slab33")
    assert (p.nx, p.ny, p.nz, p.ndir) == (33, 33, 33, 256)
    q = bench.make_problem("slab65")
    assert (q.nx, q.ndir) == (65, 1024)
