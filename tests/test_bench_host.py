"""Host logic of the benchmark (no GPU): the clock sampler's parsing of
nvidia-smi rows and the single-rank helpers."""
import bench


def test_clock_sampler_parses_rows_and_reasons():
    c = bench.ClockSampler(0)
    c.rows = [
        ["0", "2070", "2070", "900.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "1980", "2070", "1390.5", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "2070", "2070", "1100.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["garbage"],
    ]
    out = c.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_flags_thermal_slowdown():
    c = bench.ClockSampler(0)
    c.rows = [["0", "1500", "2070", "1400", "0x40", "Not Active", "Active", "Active", "Not Active"]]
    out = c.stop()
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_single_rank_environment():
    w, r, l = bench.dist_env()
    assert (w, r, l) == (1, 0, 0)
    assert bench.reduce_max(7.25, 1) == 7.25
