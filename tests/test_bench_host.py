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


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference`: one JSON line with the GPU arm's metric,
    unit, direction and config, the oracle's timing as value, cpu_baseline
    and e2e (one oracle step of the 256^3 workload, about 20 s)."""
    import json
    import os
    import subprocess
    import sys

    from paper_math_0301321_gb300 import synth
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"), "--impl",
                        "reference", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "IB steps/s" and d["higher_is_better"] is True
    assert d["config"] == bench.workload_config(synth.cochlea256(), 1)
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(None) is None
    assert capsys.readouterr().out == ""


def test_algorithmic_bytes_of_the_256_workload():
    """The per-stage byte counts behind every roofline fraction, at the 256^3
    workload's sizes (993,216 markers, 8,877 touched 8^3 tiles): each FFT pass
    reads and writes three half spectra (256 x 256 x 129 complex floats), the
    x passes add the three real fields, the x forward the force on the touched
    cells; the step's total is the figure of the bench line."""
    n, m, tiles = 256, 993216, 8877
    G = n ** 3
    spectrum = 3 * 8 * n * n * (n // 2 + 1)
    field = 3 * 4 * G
    b = {k: bench.stage_bytes(k, G, n, m, tiles) for k in
         ("keys", "sort", "records", "spread", "fft_x_fwd", "fft_y_fwd", "fft_z_proj", "fft_y_inv", "fft_x_inv",
          "interp")}
    assert b["fft_y_fwd"] == b["fft_z_proj"] == b["fft_y_inv"] == 2 * spectrum
    assert b["fft_x_inv"] == spectrum + field
    assert b["fft_x_fwd"] == field + spectrum + 3 * 4 * 512 * tiles == 458766336
    assert sum(b.values()) == 2585572000
