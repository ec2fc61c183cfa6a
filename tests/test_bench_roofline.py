"""CPU checks of the benchmark's roofline arithmetic: the FP32 peak from unit
counts and the whole-frame fraction in the method's own units (bytes = tau*36
+ rays*24, flops = pairs*F_cull + candidates*F_test) can be recomputed from
the figures the JSON line carries."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x one FMA (2 flops) per clock at 2070 MHz
    assert bench.fp32_peak_tflops(2070.0, 152) == pytest.approx(80.54784, rel=1e-12)
    assert bench.fp32_peak_tflops(1000.0, 1) == pytest.approx(0.256, rel=1e-12)


def test_frame_fraction_recomputes_from_the_lines_counters():
    # the c5 workload: 21,724,415 triangles, 8 x 128 x 4096 rays
    tau, rays = 21_724_415, 8 * 128 * 4096
    pairs, cand, frame_ms = 173_795_320, 129_623_089, 4.093
    peak, hbm = bench.fp32_peak_tflops(2070.0, 152), 6783.8
    r = bench.frame_roofline(tau, rays, pairs, cand, frame_ms, peak, hbm)
    assert r["bytes"] == tau * 36 + rays * 24 == 882_742_236
    assert r["flops"] == pairs * 200 + cand * 30
    t_alu = r["flops"] / (peak * 1e12)
    t_mem = r["bytes"] / (hbm * 1e9)
    assert r["binding"] == "alu" and t_alu > t_mem
    assert r["t_roof_ms"] == pytest.approx(1e3 * t_alu, rel=1e-12)
    assert r["frac"] == pytest.approx(r["t_roof_ms"] / frame_ms, rel=1e-12)
    assert r["achieved_tflops"] / peak == pytest.approx(r["frac"], rel=1e-12)
    assert r["achieved_gbs"] == pytest.approx(r["bytes"] / (frame_ms * 1e-3) / 1e9, rel=1e-12)


def test_frame_fraction_switches_to_hbm_when_bytes_bind():
    # few pairs and candidates against a large vertex stream: the HBM term binds
    r = bench.frame_roofline(100_000_000, 1024, 10, 10, 1.0, 80.0, 6800.0)
    assert r["binding"] == "hbm"
    assert r["t_roof_ms"] == pytest.approx(1e3 * r["bytes"] / 6800e9, rel=1e-12)
