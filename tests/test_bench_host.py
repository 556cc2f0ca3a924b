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


def test_equal_error_speedups_per_observable():
    """The speedup at equal statistical error is the ratio of 1 / (variance across chains x time):
    halving the time doubles it for every observable; doubling the spread of one flavor's n_f
    and of one G(tau) bin quarters the minimum over flavors and bins, not the others."""
    import numpy as np
    rng = np.random.default_rng(0)
    nw, nf, nb = 256, 10, 20
    acc = {"sign_sum": np.full(nw, 4.0), "obs_sum": rng.normal(1.0, 0.1, (nw, 3 * 5 + 1 + 36)),
           "order_sum": rng.normal(2.0, 0.1, (nw, nf)), "g_tau": rng.normal(0.5, 0.05, (nw, nf, nb))}
    est = bench.chain_estimates(acc, 5, 50.0, nb)
    assert est["n_f"].shape == (nw, nf) and est["G_tau"].shape == (nw, nb)
    assert np.allclose(est["docc"], acc["obs_sum"][:, 10:15].mean(1) / 4.0)
    sp = bench.speedups(bench.efficiencies(est, 1.0), bench.efficiencies(est, 2.0))
    assert all(abs(v - 2.0) < 1e-12 for v in sp.values())
    wide = {k: v.copy() for k, v in est.items()}
    wide["n_f"][:, 3] = 2.0 * (wide["n_f"][:, 3] - wide["n_f"][:, 3].mean())
    wide["G_tau"][:, 7] = 2.0 * (wide["G_tau"][:, 7] - wide["G_tau"][:, 7].mean())
    sp = bench.speedups(bench.efficiencies(wide, 1.0), bench.efficiencies(est, 1.0))
    assert abs(sp["n_f_min_over_flavors"] - 0.25) < 1e-12 and abs(sp["G_tau_min_over_bins"] - 0.25) < 1e-12
    assert sp["docc"] == 1.0 and abs(sp["G_tau_median_over_bins"] - 1.0) < 1e-12
    # orbital occupations sum the two spins of each orbital (flavor f = 2a + s)
    assert est["n_orbital"].shape == (nw, 5)
    assert np.allclose(est["n_orbital"][:, 2], est["n_f"][:, 4] + est["n_f"][:, 5])
    # pooled over bins: one wider bin of twenty raises the summed variance, not four-fold
    vb = est["G_tau"].var(axis=0, ddof=1)
    want = vb.sum() / (vb.sum() + 3.0 * vb[7])
    assert abs(sp["G_tau_pooled"] - want) < 1e-12 and 0.25 < sp["G_tau_pooled"] < 1.0
