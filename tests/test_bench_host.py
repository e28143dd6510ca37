"""Host helpers of the benchmark (no GPU): clock-sample parsing and the
algorithmic byte count of one pull iteration."""
import types

import pytest

import bench


def test_parse_clocks_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.1, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "[N/A] garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.parse_clocks(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}


def test_parse_clocks_flags_thermal_and_empty():
    c = bench.parse_clocks(["0, 1500, 2070, 1000, 0x40, Not Active, Active, Not Active, Not Active"])
    assert c["reasons"] == ["hw_thermal_slowdown"] and c["sm_mhz"] == 1500.0
    assert bench.parse_clocks([]) is None


@pytest.mark.parametrize("sr,s_w,s_f,extra", [("tropical", 0.0, 4.0, 0.0), ("real", 4.0, 4.0, 0.0),
                                               ("boolean", 0.125, 0.125, 0.0), ("selmax", 4.0, 4.0, 4.0)])
def test_iteration_bytes_terms(sr, s_w, s_f, extra):
    # 10 active chunks of C = 32 rows with 5,000 slots, 300 new vertices, n = 100,000
    it = types.SimpleNamespace(slots=5000, active_chunks=10, frontier=300)
    want = 4 * 5000 + 8 * 10 + 320 * (4 + s_w) + 300 * (8 + extra) + 100000 * s_f
    assert bench.iteration_bytes(it, sr, 100000, 32) == pytest.approx(want)
    idle = types.SimpleNamespace(slots=0, active_chunks=0, frontier=0)  # only the vector pass
    assert bench.iteration_bytes(idle, sr, 100000, 32) == pytest.approx(100000 * s_f)
