"""The bench's FP32 roofline arithmetic on a hand-made launch list (no GPU)."""

import math
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def _launch(kind, states, g1=0, g2=0, d1=0, d2=0, reductions=0, spawned=0):
    return {"kind": kind, "states": states, "g1": g1, "g2": g2, "d1": d1, "d2": d2, "reductions": reductions,
            "spawned": spawned}


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
