"""The roofline arithmetic of bench.py on synthetic profiler records (CPU)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6787.9, "bf16_tflops": 1874.8, "bf16_tflops_sustained": 1703.3}


def test_tensor_family_against_the_sustained_tf32_peak():
    # 1.1e15 algorithmic flops in 2000 ms: 550 TFLOP/s
    r = bench.roofline_of("tensor", {"ms": 2000.0, "flops": 1.1e15, "bytes": 0.0, "launches": 10},
                          PEAKS, "measured", 1)
    peak = 1703.3 * 1.1 / 2.25
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(550.0)
    assert r["peak"] == pytest.approx(peak)
    assert r["frac"] == pytest.approx(550.0 / peak)
    assert r["tensor_pipe_frac"] == pytest.approx(3 * 550.0 / peak)
    assert r["traffic"] == pytest.approx(bench.TC_CORNER_DRAM_BYTES)


def test_alu_and_hbm_families():
    rec = {"ms": 1000.0, "flops": 1.0e12, "bytes": 3.0e12, "launches": 5}
    f64 = bench.roofline_of("svd", rec, PEAKS, "measured", 1)
    assert f64["bound"] == "alu" and f64["frac"] == pytest.approx(1.0 / bench.FP64_NOMINAL_TFLOPS)
    assert bench.roofline_of("contract", rec, PEAKS, "measured", 0)["peak"] == bench.FP64_NOMINAL_TFLOPS
    f32 = bench.roofline_of("contract", rec, PEAKS, "measured", 1)
    assert f32["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    hbm = bench.roofline_of("other", rec, PEAKS, "measured", 1)
    assert hbm["bound"] == "hbm" and hbm["unit"] == "GB/s"
    assert hbm["achieved"] == pytest.approx(3000.0) and hbm["frac"] == pytest.approx(3000.0 / 6787.9)
