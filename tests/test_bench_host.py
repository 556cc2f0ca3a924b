"""CPU tests of bench.py's host logic: the clock record taken during the timed region,
the Krylov-dimension histogram and the tie between the traffic record and the kernel
sources."""
import json

import bench


def clock_record(lines):
    s = bench.ClockSampler(0)
    s.f.write("".join(l + "\n" for l in lines))
    s.t0 = 0.0
    return s.stop()


def test_clock_record_median_max_and_reasons():
    row = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {cap}"
    d = clock_record([row.format(sm=2070, hw="Not Active", cap="Not Active"),
                      row.format(sm=1965, hw="Not Active", cap="Active"),
                      row.format(sm=2070, hw="Not Active", cap="Not Active")])
    assert d["sm_mhz"] == 2070 and d["sm_max_mhz"] == 2070 and d["samples"] == 3
    assert d["reasons"] == ["sw_power_cap"]
    d = clock_record([row.format(sm=1500, hw="Active", cap="Not Active")])
    assert d["reasons"] == ["hw_slowdown"] and d["sm_mhz"] == 1500


def test_clock_record_without_samples():
    d = clock_record(["garbage"])
    assert d["samples"] == 0 and d["sm_mhz"] is None and d["reasons"] == ["nvidia-smi unavailable"]


def test_trim_hist_drops_empty_bins_and_marks_the_last():
    assert bench.trim_hist([0, 5, 0, 7, 2]) == {"1": 5, "3": 7, ">=4": 2}
    assert bench.trim_hist([0, 0]) == {}


def test_traffic_record_needs_the_current_sources(tmp_path, monkeypatch):
    sha = bench.source_sha()
    assert len(sha) == 16
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "items_kernel_traffic.json").write_text(json.dumps({"source_sha": sha, "dram_bytes_per_launch": 123}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic(sha) == 123
    assert bench.measured_traffic("0" * 16) is None
