"""The bench's FP32 roofline arithmetic on a hand-made launch list (no GPU)."""

import math
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def _launch(kind, states, g1=0, g2=0, d1=0, d2=0, reductions=0, spawned=0, algorithmic_bytes=0.0):
    return {"kind": kind, "states": states, "g1": g1, "g2": g2, "d1": d1, "d2": d2, "reductions": reductions,
            "spawned": spawned, "algorithmic_bytes": algorithmic_bytes}


def test_fp32_roofline_counts_flops_of_the_selected_launches():
    launches = [
        _launch("fill", 0),
        _launch("pass", 3, g1=2, g2=1, d2=3, reductions=1),        # 3 * (32 + 32 + 18 + 16) = 294 per amplitude
        _launch("pass", 1, g1=5, spawned=3),                       # not selected (one state)
        _launch("pass", 3, g1=1, d1=1, reductions=2, spawned=9),   # 3 * (16 + 6 + 32) + 16 * 9 = 306
        _launch("finish", 0),
    ]
    n = 10
    stats = {"launches": 6, "total_ms": 2.0}   # three calls of the two selected launches
    r = bench.fp32_roofline(launches, stats, n, True, 2000.0)
    flops_call = 2 ** n * (294 + 306)
    assert math.isclose(r["flops_per_launch"], flops_call / 2)
    assert math.isclose(r["achieved"], flops_call * 3 / 2e-3 / 1e12)
    assert math.isclose(r["peak"], 152 * 128 * 2 * 2000e6 / 1e12)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"])
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    single = bench.fp32_roofline(launches, {"launches": 3, "total_ms": 1.0}, n, False, 2000.0)
    assert math.isclose(single["flops_per_launch"], 2 ** n * (5 * 16 + 16 * 3))
    assert bench.fp32_roofline(launches, {"launches": 0, "total_ms": 0.0}, n, True, 2000.0) is None


def test_combined_bound_takes_the_larger_bound_of_each_launch():
    n = 20
    dim = 2 ** n
    # one memory-bound launch (few flops, many bytes) and one arithmetic-bound launch
    mem = _launch("pass", 3, g1=1, algorithmic_bytes=48.0 * dim)          # 48 flops / amplitude
    ari = _launch("pass", 3, g1=40, algorithmic_bytes=48.0 * dim)         # 1920 flops / amplitude
    hbm, mhz = 5000.0, 2000.0
    peak = 152 * 128 * 2 * mhz * 1e6
    t_mem = max(48.0 * dim / (hbm * 1e9), 48.0 * dim / peak)
    t_ari = max(48.0 * dim / (hbm * 1e9), 1920.0 * dim / peak)
    assert t_mem == 48.0 * dim / (hbm * 1e9) and t_ari == 1920.0 * dim / peak
    measured_ms = 2 * 1000.0 * (t_mem + t_ari) / 0.8     # two calls at 0.8 of the combined bound
    r = bench.fp32_roofline([mem, ari], {"launches": 4, "total_ms": measured_ms}, n, True, mhz, hbm)
    assert math.isclose(r["combined_bound_frac"], 0.8)
    assert "combined_bound_frac" not in bench.fp32_roofline([mem, ari], {"launches": 4, "total_ms": 1.0}, n, True, mhz)
