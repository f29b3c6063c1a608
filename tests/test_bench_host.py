"""Host logic of bench.py that needs no GPU: the clock record and the peaks file."""
import bench


def sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_clock_summary_median_max_and_reasons():
    idle = "0, {sm}, 2070, 850.1, 0x0000000000000000, Not Active, Not Active, Not Active, {cap}"
    lines = [idle.format(sm=v, cap="Not Active") for v in (2070, 1980, 2070, 2055)]
    lines.append(idle.format(sm=1965, cap="Active"))
    lines.append("garbage")                       # short lines are skipped
    lines.append("0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active")
    out = sampler(lines).summary()
    assert out["sm_mhz"] == 2055.0                # median of 1965, 1980, 2055, 2070, 2070
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 5


def test_clock_summary_names_each_slowdown():
    row = "0, 1500, 2070, 1300.0, 0x8, {a}, {b}, {c}, Not Active"
    out = sampler([row.format(a="Active", b="Not Active", c="Not Active"),
                   row.format(a="Not Active", b="Active", c="Active")]).summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples_says_so():
    out = sampler([]).summary()
    assert out["sm_mhz"] is None and out["reasons"] == ["clocks not sampled"]


def test_peaks_are_the_measured_ones_when_present():
    pk, kind = bench.peaks()
    assert pk["hbm_gbs"] > 0
    assert kind in ("measured", "fallback")
