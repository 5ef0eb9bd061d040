"""The measurement script's roofline arithmetic on the CPU: the work counts
behind `roofline.frac` (the method's 5 flop per row and fine step for F, the
FP64 flop per point of the CGC steps (a)-(c), algorithmic bytes for the FP32
defect CGC), the derived FP32 roof, and the fine kernel's measured traffic
following the layout the autotuner picked."""
import math
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

W = SimpleNamespace(dim=1, reaction_kind=0, N=64, nx=1023, advection=0)
UNITS = {"row_steps": 4096 * 64 * 1024 * 64, "points": 4096 * 64 * 1023}


def test_fp32_roof_is_sms_lanes_fma_clock():
    assert bench.FP32_ALU_PEAK == pytest.approx(152 * 128 * 2 * 2.070e9 / 1e12)


def test_fine_roofline_counts_five_flop_per_row_step():
    ms, launches = 100.0, 4
    e = bench.roofline_entry("fine", ms, launches, UNITS, "mixed", W, 7000.0, "measured")
    ach = 5.0 * UNITS["row_steps"] / (ms / 1e3) / 1e12
    assert e["bound"] == "alu" and e["unit"] == "TFLOP/s"
    assert e["achieved"] == pytest.approx(ach)
    assert e["frac"] == pytest.approx(ach / bench.FP32_ALU_PEAK)
    e64 = bench.roofline_entry("fine", ms, launches, UNITS, "fp64", W, 7000.0, "measured")
    assert e64["frac"] == pytest.approx(ach / bench.FP64_ALU_PEAK)


@pytest.mark.parametrize("cls,per_pt", [("cgc_fwd", 2.5 * 6 + 1 + 1),
                                        ("cgc_solve", 22.0 * 33 / 64),
                                        ("cgc_inv", 2.5 * 6 + 4)])
def test_fp64_cgc_counts_per_point(cls, per_pt):
    ms = 50.0
    e = bench.roofline_entry(cls, ms, 1, UNITS, "mixed", W, 7000.0, "measured")
    assert e["bound"] == "alu" and e["peak"] == bench.FP64_ALU_PEAK
    assert e["achieved"] == pytest.approx(per_pt * UNITS["points"] / (ms / 1e3) / 1e12)
    # the all-FP64 forward also forms the jump (I + dT A) F - prev: 7 flop
    if cls == "cgc_fwd":
        e64 = bench.roofline_entry(cls, ms, 1, UNITS, "fp64", W, 7000.0, "measured")
        assert e64["achieved"] == pytest.approx((2.5 * 6 + 1 + 7) * UNITS["points"]
                                                / (ms / 1e3) / 1e12)


def test_defect_cgc_is_counted_in_bytes():
    ms, peak = 20.0, 7000.0
    K = 33
    spec = 8 * K / 64
    e = bench.roofline_entry("cgc_fwd", ms, 1, UNITS, "mixed_defect", W, peak, "measured")
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert e["achieved"] == pytest.approx((28 + spec) * UNITS["points"] / (ms / 1e3) / 1e9)
    assert e["frac"] == pytest.approx(e["achieved"] / peak)
    s = bench.roofline_entry("cgc_solve", ms, 1, UNITS, "mixed_defect", W, peak, "measured")
    assert s["achieved"] == pytest.approx(4 * spec * UNITS["points"] / (ms / 1e3) / 1e9)


def test_fine_traffic_follows_the_tuned_layout():
    key = "NVIDIA GB300|fine32|nx=1023|N=64|J=64"
    times = {key + "|ms@S=512": "L4R32:0.83 P1R32:0.79"}
    table = bench.MEASURED_FINE_TRAFFIC_B_PER_POINT
    assert bench.fine_traffic_per_point({key: "P1R32", **times}) == table["P"]
    assert bench.fine_traffic_per_point({key: "L4R32", **times}) == table["L"]
    # layouts without a capture, no choice, or several choices: no figure
    assert bench.fine_traffic_per_point({key: "W2R16", **times}) is None
    assert bench.fine_traffic_per_point(times) is None
    other = "NVIDIA GB300|fine32|nx=511|N=64|J=64"
    assert bench.fine_traffic_per_point({key: "P1R32", other: "L4R16"}) is None
    # the per-point figures are the captured bytes of one 512-sample launch
    assert table["P"] * 512 * 64 * 1023 == pytest.approx(243.6e6)
    assert math.isclose(table["L"] * 512 * 64 * 1023, 247.7e6)


def test_traffic_scales_by_points_per_launch():
    pts, launches = 1_000_000, 4
    per = bench.MEASURED_TRAFFIC_B_PER_POINT["mixed"]["cgc_inv"]
    assert bench.traffic_per_launch("cgc_inv", "mixed", pts, launches) == pytest.approx(
        per * pts / launches)
    assert bench.traffic_per_launch("cgc_inv", "fp64", pts, launches) is None
