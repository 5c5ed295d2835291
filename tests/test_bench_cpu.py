"""Host-side checks of bench.py that need no GPU: the per-class table, the
algorithmic flops per step and the roofline object of the JSON line are the
arithmetic the contract states (achieved = algorithmic work per launch over
the launch's average duration, frac = achieved / peak), on synthetic kernel
statistics."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

KSTATS = [
    # 3 profiled steps: 4 sector-product launches per step, 2 element-wise
    {"name": "sector_gemm_kernel", "launches": 12, "ms": 7.5, "bytes": 12e9, "flops": 6.9e9},
    {"name": "layout:scatter", "launches": 6, "ms": 1.8, "bytes": 17e9, "flops": 0.0},
    {"name": "propagate_kernel", "launches": 6, "ms": 0.6, "bytes": 3.4e9, "flops": 0.0},
]
PEAKS = {"fp64_tflops": {"burst": 1.1}, "hbm_gbs": 7000.0}


def test_class_table_shares_and_rates():
    t = bench.class_table(KSTATS, 3)
    assert [r["name"] for r in t] == ["sector_gemm_kernel", "layout:scatter", "propagate_kernel"]
    assert sum(r["share"] for r in t) == pytest.approx(1.0)
    top = t[0]
    assert top["launches_per_step"] == 4 and top["ms_per_step"] == pytest.approx(2.5)
    assert top["TFLOP_per_s"] == pytest.approx(6.9e9 / 7.5e-3 / 1e12)
    assert top["GB_per_s"] == pytest.approx(12e9 / 7.5e-3 / 1e9)
    assert t[1]["TFLOP_per_s"] is None


def test_flops_per_step_sums_the_contraction_classes():
    assert bench.gemm_flops_per_step(KSTATS, 3) == pytest.approx(6.9e9 / 3)


def test_roofline_of_the_dominant_class():
    r = bench.roofline_sparse(KSTATS, 3, PEAKS)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["kernel"] == "sector_gemm_kernel"
    assert r["achieved"] == pytest.approx(6.9e9 / 7.5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.1)
    assert r["avg_launch_ms"] == pytest.approx(7.5 / 12)
    assert r["algorithmic_flops_per_launch"] * r["launches_per_step"] * 3 == pytest.approx(6.9e9)
    assert r["traffic"] is None
    # an element-wise class on top is measured against the copy bandwidth
    hbm = bench.roofline_sparse([dict(KSTATS[1], ms=9.0)] + KSTATS[2:], 3, PEAKS)
    assert hbm["bound"] == "hbm" and hbm["unit"] == "GB/s"
    assert hbm["frac"] == pytest.approx(17e9 / 9e-3 / 1e9 / 7000.0)
