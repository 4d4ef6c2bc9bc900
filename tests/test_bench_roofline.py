"""The benchmark line's roofline objects can be recomputed from their own
fields: achieved = per-unit work x units per launch / launch time, frac =
achieved / peak, peak = lanes per clock per SM x SMs x clock (CPU only)."""
import math

import bench


RATES = [{"ex2": 32.0, "ffma": 123.6, "ffma2": 125.8, "clock_mhz": 2050.0},
         {"ex2": 32.0, "ffma": 123.6, "ffma2": 125.8, "clock_mhz": 2040.0}]
NCU = {"bytes_per_launch": 1.0e8, "fma_pipe_active": 0.6, "issue_active": 0.62,
       "xu_active": 0.13, "fp32_lane_ops": 1.4e10}


def test_fp32_roofline_follows_from_its_fields():
    out = bench.roofline_fields(1.8e8, 8.6e8, 6.2e-4, RATES, 152, 2070.0, NCU)
    r = out["roofline"]
    pu = r["per_unit"]
    achieved = pu["fp32_lane_ops"] * pu["units_per_launch"] / (pu["launch_ms"] / 1e3) / 1e12
    assert math.isclose(r["achieved"], achieved, rel_tol=1e-9)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-9)
    assert math.isclose(r["peak"], 123.6 * 152 * 2045.0 * 1e6 / 1e12, rel_tol=1e-9)
    assert r["traffic"] == 1.0e8 and r["bound"] == "alu"
    assert pu["fp32_lane_ops"] == bench.FP32_OPS_PER_PAIR


def test_ex2_rooflines_count_two_per_pair():
    out = bench.roofline_fields(1.8e8, 8.6e8, 6.2e-4, RATES, 152, 2070.0, None)
    e = out["roofline_ex2"]
    peak = 32.0 * 152 * 2045.0 * 1e6
    for key, pairs in (("in_range", 1.8e8), ("listed", 8.6e8)):
        assert math.isclose(e[key]["achieved"], 2 * pairs / 6.2e-4 / 1e9, rel_tol=1e-9)
        assert math.isclose(e[key]["frac"], 2 * pairs / 6.2e-4 / peak, rel_tol=1e-9)
        assert math.isclose(e[key]["frac"], e[key]["achieved"] / e[key]["peak"], rel_tol=1e-9)
    assert out["fp32_executed"] is None and out["roofline"]["traffic"] is None


def test_executed_fp32_uses_the_counted_work():
    out = bench.roofline_fields(1.8e8, 8.6e8, 6.2e-4, RATES, 152, 2070.0, NCU)
    x = out["fp32_executed"]
    assert math.isclose(x["per_in_range_pair"], 1.4e10 / 1.8e8, rel_tol=1e-12)
    assert math.isclose(x["frac"], x["achieved"] / out["roofline"]["peak"], rel_tol=1e-9)


def test_fallback_clock_without_live_rates():
    out = bench.roofline_fields(1.0e8, 5.0e8, 1e-3, [], 152, 1900.0, None)
    assert math.isclose(out["roofline"]["peak"], 128.0 * 152 * 1900.0 * 1e6 / 1e12, rel_tol=1e-9)
    assert "fallback" in out["roofline"]["peak_basis"]
