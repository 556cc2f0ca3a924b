"""Batched CT-HYB chains (kt_sweep) against the oracle chain (oracle/ctqmc.py).

With the same uniforms, the FP64 path takes the same Metropolis decisions as the
oracle, whose weights are recomputed from scratch every step: the final
configurations must be identical operator by operator (times bit for bit: both
sides round t1 = u2 beta and t2 = t1 + u3 l as written). A decision can only
differ where u5 lies within the ratio's rounding error of the acceptance
probability (about 1e-12 relative in FP64); the seeds below have none.
The tracked weights (trace sign and log, sum of log|det|, sign of w) must match the
from-scratch values of the final configurations; the measured G(tau) sums, orders
and observables at beta/2 must match the oracle's accumulators.
Without interaction, G(tau) must be the semicircular one (statistical, 5 standard
errors over independent walkers).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle.ctqmc import Hyb, chain, weight  # noqa: E402
from oracle.oracle import Model, Params  # noqa: E402
from paper_0908_0681_gb300 import engine, kt, workloads  # noqa: E402
from tests import parity  # noqa: E402


def model_pair(spec, precision):
    P = Params(spec.n_orb, spec.U, spec.J, Up=spec.up, mu=spec.mu, delta=spec.delta, beta=spec.beta,
               trunc_eps=spec.trunc_eps, deg_tol=spec.deg_tol)
    return Model(P), engine.model_from_spec(spec, precision=precision)


def run_both(spec, nw, steps, k_cap, n_bins, meas_every, seed, precision=kt.KT_FP64, observables=True,
             cache_ops=0):
    om, gm = model_pair(spec, precision)
    table = workloads.semicircular_hybridization(spec.beta, 2 * spec.n_orb, n_tau=2000)
    u = workloads.sweep_uniforms(steps, nw, seed=seed)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=k_cap, n_bins=n_bins, measure_obs=observables,
                      cache_ops=cache_ops)
    sw.run(torch.as_tensor(u, device="cuda"), meas_every=meas_every)
    ref = chain(om, Hyb(table, spec.beta), [[] for _ in range(nw)], u, k_cap=k_cap, n_bins=n_bins,
                meas_every=meas_every, observables=observables)
    return om, Hyb(table, spec.beta), sw, ref


@pytest.mark.parametrize("k_cap,cache_ops", [(64, 0), (2, 0), (64, 64), (64, 12)])
def test_three_orbital_chain_matches_oracle(k_cap, cache_ops):
    """cache_ops > 0: the ratios come from the partial-state cache; with 12 the walkers
    move in and out of the cached length."""
    w = workloads.three_orbital()
    spec = w.model
    nw, steps = 16, 400
    om, hyb, sw, ref = run_both(spec, nw, steps, k_cap, n_bins=20, meas_every=8, seed=21, cache_ops=cache_ops)
    cnt = sw.counters()
    acc = ref["accepted"]
    assert cnt["trace_errors"] == 0
    assert cnt["insert_accepted"] + cnt["remove_accepted"] == int((acc == 1).sum())
    assert cnt["insert_proposed"] + cnt["remove_proposed"] == nw * steps
    if k_cap == 2:
        assert cnt["refused_at_k_cap"] > 0
    cfg = sw.configs()
    for i in range(nw):
        assert cfg[i] == ref["configs"][i], i
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    assert (st["sign"] == ref["sign"]).all() and (st["trace_sign"] == ref["trace_sign"]).all()
    assert np.abs(st["trace_logabs"] - ref["trace_log"]).max() < 1e-9
    det_ref = ref["logw"] - ref["trace_log"]
    assert np.abs(st["det_logabs"] - det_ref).max() < 1e-8
    for i in range(nw):
        orders = [sum(1 for t, f, d in cfg[i] if f == g and d == 1) for g in range(2 * spec.n_orb)]
        assert list(st["order"][i]) == orders
    a = {k: v.cpu().numpy() for k, v in sw.accumulators().items()}
    assert np.allclose(a["sign_sum"], ref["sign_sum"])
    assert np.allclose(a["order_sum"], ref["order_sum"])
    assert np.abs(a["g_tau"] - ref["g_acc"]).max() <= 1e-9 * max(1.0, np.abs(ref["g_acc"]).max())
    assert np.abs(a["obs_sum"] - ref["obs_sum"]).max() <= 1e-8


def test_five_orbital_fp32_chain_weights():
    """FP32-Krylov traces in the chain: the tracked weights of the final configurations
    against the oracle's from-scratch weights (trace within the FP32 tolerance)."""
    w = workloads.five_orbital_sweep(beta=10.0)
    spec = w.model
    om, gm = model_pair(spec, kt.KT_FP32_KRYLOV)
    nw, steps = 64, 300
    table = workloads.semicircular_hybridization(spec.beta, 10, n_tau=2000)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=20)
    sw.run(torch.as_tensor(workloads.sweep_uniforms(steps, nw, seed=5), device="cuda"), meas_every=10)
    cnt = sw.counters()
    assert cnt["trace_errors"] == 0 and cnt["insert_accepted"] > 0 and cnt["remove_accepted"] > 0
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    hyb = Hyb(table, spec.beta)
    for i, ops in enumerate(sw.configs()):
        s, lw, sT, lT = weight(om, hyb, ops)
        assert s == st["sign"][i] and sT == st["trace_sign"][i], i
        assert abs(math.expm1(st["trace_logabs"][i] - lT)) < 1e-5, i
        assert abs(st["det_logabs"][i] - (lw - lT)) < 1e-8, i


def test_semicircular_green_function_without_interaction():
    """One orbital, U = 0, mu = 0: G(tau) = -F(tau) (Bethe lattice, t = 1)."""
    beta, nw, steps, nb = 8.0, 512, 3000, 16
    spec = workloads.ModelSpec(1, 0.0, 0.0, mu=0.0, delta=(0.0,), beta=beta, trunc_eps=0.0)
    gm = engine.model_from_spec(spec, precision=kt.KT_FP64)
    table = workloads.semicircular_hybridization(beta, 2, n_tau=2000)
    sw = engine.Sweep(gm, table, beta, nw, k_cap=64, n_bins=nb)
    u = torch.rand((steps, nw, 6), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    sw.run(u[:500])                   # warm-up
    sw.reset_accumulators()
    sw.run(u[500:], meas_every=10)
    a = {k: v.cpu().numpy() for k, v in sw.accumulators().items()}
    assert (a["sign_sum"] > 0).all()
    gw = (a["g_tau"] * (nb / beta ** 2) / a["sign_sum"][:, None, None]).mean(axis=1)   # [nw, nb]
    mean, err = gw.mean(0), gw.std(0, ddof=1) / math.sqrt(nw)
    grid = np.linspace(0, beta, 2001)
    exact = np.array([-np.mean(np.interp(np.linspace(b * beta / nb, (b + 1) * beta / nb, 201), grid, table[0]))
                      for b in range(nb)])
    assert np.all(np.abs(mean - exact) < 5 * err + 1e-3), (mean, exact, err)


def test_set_configs_restart_matches_oracle():
    """Chains started from given configurations: the from-scratch weights (host inverses,
    device traces) equal the oracle's, and the continued chains match the oracle chain."""
    w = workloads.three_orbital()
    spec = w.model
    om, gm = model_pair(spec, kt.KT_FP64)
    table = workloads.semicircular_hybridization(spec.beta, 6, n_tau=2000)
    hyb = Hyb(table, spec.beta)
    cand = workloads.generate_sequences(w, 400, seed=9)
    keep = []
    for i in range(cand.n):
        ops = list(zip(*[a.tolist() for a in cand.walker(i)]))
        if max([sum(1 for t, f, d in ops if f == g and d == 1) for g in range(6)] + [0]) <= 8 and weight(om, hyb, ops)[0] != 0:
            keep.append(i)
        if len(keep) == 16:
            break
    assert len(keep) == 16
    seqs = cand.subset(keep)
    init = [list(zip(*[a.tolist() for a in seqs.walker(i)])) for i in range(seqs.n)]
    sw = engine.Sweep(gm, table, spec.beta, 16, k_cap=16, n_bins=10)
    sw.set_configs(seqs)
    assert sw.configs() == init
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    for i, ops in enumerate(init):
        s, lw, sT, lT = weight(om, hyb, ops)
        assert s == st["sign"][i] and sT == st["trace_sign"][i]
        assert abs(st["trace_logabs"][i] - lT) < 1e-9 and abs(st["det_logabs"][i] - (lw - lT)) < 1e-9
    u = workloads.sweep_uniforms(200, 16, seed=33)
    sw.run(torch.as_tensor(u, device="cuda"), meas_every=0)
    ref = chain(om, hyb, init, u, k_cap=16)
    assert sw.configs() == ref["configs"]
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    assert (st["sign"] == ref["sign"]).all()
    assert np.abs(st["det_logabs"] - (ref["logw"] - ref["trace_log"])).max() < 1e-8
    # a malformed batch (a flavor with two c^+ in a row) is refused and the chains restart empty
    bad = workloads.Sequences(np.array([0, 2] + [2] * 15, np.int32), np.array([1.0, 2.0]), np.array([0, 0], np.uint8),
                              np.array([1, 1], np.uint8))
    with pytest.raises(kt.KtError):
        sw.set_configs(bad)
    assert all(len(c) == 0 for c in sw.configs())


def test_refresh_keeps_the_oracle_chain():
    """Drift guard (kt_sweep_refresh): three-orbital FP64 chains refreshed from scratch every
    100 steps (M, log|det|, permutation sign and trace recomputed on the device) take the
    oracle chain's decisions for 400 steps; the deviations the refresh reports are at FP64
    rounding, and the refreshed values equal the oracle's weights."""
    w = workloads.three_orbital()
    spec = w.model
    nw, steps, k_cap = 16, 400, 64
    om, gm = model_pair(spec, kt.KT_FP64)
    table = workloads.semicircular_hybridization(spec.beta, 2 * spec.n_orb, n_tau=2000)
    hyb = Hyb(table, spec.beta)
    u = workloads.sweep_uniforms(steps, nw, seed=41)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=k_cap, n_bins=10)
    ut = torch.as_tensor(u, device="cuda")
    devs = []
    for b in range(4):
        sw.run(ut[b * 100:(b + 1) * 100].contiguous())
        devs.append(sw.refresh())
    ref = chain(om, hyb, [[] for _ in range(nw)], u, k_cap=k_cap)
    assert sw.configs() == ref["configs"]
    for d in devs:
        assert d["sign_mismatches"] == 0 and d["unchanged"] == 0
        assert d["trace_log"] < 1e-9 and d["det_log"] < 1e-9, d
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    for i, ops in enumerate(sw.configs()):
        s, lw, sT, lT = weight(om, hyb, ops)
        assert s == st["sign"][i] and sT == st["trace_sign"][i]
        assert abs(st["trace_logabs"][i] - lT) < 1e-9
        assert abs(st["det_logabs"][i] - (lw - lT)) < 1e-10
    # the refreshed inverse matrices carry the chain on: 100 more steps still match the oracle
    u2 = workloads.sweep_uniforms(100, nw, seed=42)
    sw.run(torch.as_tensor(u2, device="cuda"))
    ref2 = chain(om, hyb, ref["configs"], u2, k_cap=k_cap)
    assert sw.configs() == ref2["configs"]


def test_refresh_bounds_fp32_drift():
    """Five orbitals at beta = 50, FP32 traces, 400 steps from thermalised configurations:
    the tracked trace is a product of accepted FP32 ratios and drifts; after the refresh every
    tracked trace is a fresh evaluation, within RTOL of the oracle's."""
    nw, steps, beta = 64, 400, 50.0
    spec, table, seqs = _thermal_five_orbital(nw, beta, seed=13)
    gm = engine.model_from_spec(spec, precision=kt.KT_FP32_KRYLOV)
    sw = engine.Sweep(gm, table, beta, nw, k_cap=128, n_bins=10)
    sw.set_configs(seqs)
    # a uniform stream of its own: the thermalisation used seed 14, and replaying it would propose
    # operators at exactly the times it inserted (ties of measure zero that the oracle's permutation
    # sign orders differently)
    sw.run(torch.as_tensor(workloads.sweep_uniforms(steps, nw, seed=1013), device="cuda"))
    cnt = sw.counters()
    n_acc = cnt["insert_accepted"] + cnt["remove_accepted"]
    d = sw.refresh()
    assert d["sign_mismatches"] == 0 and d["unchanged"] == 0
    assert d["det_log"] < 1e-8 and d["trace_log"] <= n_acc * parity.RATIO_RTOL[kt.KT_FP32_KRYLOV], d
    om, _ = model_pair(spec, kt.KT_FP64)
    hyb = Hyb(table, beta)
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    for i, ops in enumerate(sw.configs()):
        s, lw, sT, lT = weight(om, hyb, ops)
        assert s == st["sign"][i] and sT == st["trace_sign"][i], i
        assert abs(math.expm1(st["trace_logabs"][i] - lT)) <= parity.RTOL[kt.KT_FP32_KRYLOV], i
        assert abs(st["det_logabs"][i] - (lw - lT)) < 1e-8, i


@pytest.mark.parametrize("precision", [kt.KT_FP64, kt.KT_FP32_KRYLOV])
def test_seven_orbital_chain_weights(precision):
    """Seven orbitals (36-row kernel blocks, N_tr = 63) with the semicircular bath of bandwidth
    2: after 200 steps every chain's determinants match the oracle's, its trace evaluated
    from scratch by the library matches the oracle's within RTOL, and the tracked trace (a
    product of the accepted ratios) stays within the accepted moves' accumulated ratio bound
    of it."""
    w = workloads.seven_orbital()
    spec = w.model
    om, gm = model_pair(spec, precision)
    nw, steps = 32, 200
    table = workloads.semicircular_hybridization(spec.beta, 14, n_tau=2000, half_bandwidth=1.0)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=32, n_bins=10)
    sw.run(torch.as_tensor(workloads.sweep_uniforms(steps, nw, seed=7), device="cuda"))
    cnt = sw.counters()
    assert cnt["trace_errors"] == 0 and cnt["insert_accepted"] > 0
    n_acc = cnt["insert_accepted"] + cnt["remove_accepted"]
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    cfg = sw.configs()
    offs = np.cumsum([0] + [len(c) for c in cfg]).astype(np.int32)
    flat = [op for c in cfg for op in c]
    seqs = workloads.Sequences(offs, np.array([o[0] for o in flat], np.float64), np.array([o[1] for o in flat], np.uint8),
                               np.array([o[2] for o in flat], np.uint8))
    fresh_s, fresh_l, fresh_st = (t.cpu().numpy() for t in engine.trace(gm, engine.DeviceSeqs.from_host(seqs)))
    assert (fresh_st == kt.KT_OK).all()
    hyb = Hyb(table, spec.beta)
    rtol = parity.RTOL[precision]
    for i, ops in enumerate(cfg):
        s, lw, sT, lT = weight(om, hyb, ops)
        assert s == st["sign"][i] and sT == st["trace_sign"][i] == fresh_s[i], i
        assert abs(math.expm1(fresh_l[i] - lT)) <= rtol, i
        assert abs(math.expm1(st["trace_logabs"][i] - fresh_l[i])) <= n_acc * parity.RATIO_RTOL[precision] + rtol, i
        assert abs(st["det_logabs"][i] - (lw - lT)) < 1e-8, i


def test_five_orbital_fp64_chain_matches_oracle_from_given_configs():
    """The bench's model (five orbitals, beta 50, semicircular bath), chains started from
    Poisson(6) configurations: the FP64 chain reaches the oracle chain's configurations."""
    w = workloads.five_orbital()
    spec = w.model
    om, gm = model_pair(spec, kt.KT_FP64)
    table = workloads.semicircular_hybridization(spec.beta, 10, n_tau=2000)
    hyb = Hyb(table, spec.beta)
    cand = workloads.generate_sequences(w, 64, seed=12)
    keep = [i for i in range(cand.n) if weight(om, hyb, list(zip(*[a.tolist() for a in cand.walker(i)])))[0] != 0][:12]
    seqs = cand.subset(keep)
    init = [list(zip(*[a.tolist() for a in seqs.walker(i)])) for i in range(seqs.n)]
    nw, steps = len(init), 60
    u = workloads.sweep_uniforms(steps, nw, seed=13)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=10)
    sw.set_configs(seqs)
    sw.run(torch.as_tensor(u, device="cuda"))
    ref = chain(om, hyb, init, u, k_cap=64)
    assert sw.configs() == ref["configs"]
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    assert (st["sign"] == ref["sign"]).all()
    assert np.abs(st["trace_logabs"] - ref["trace_log"]).max() < 1e-8
    assert np.abs(st["det_logabs"] - (ref["logw"] - ref["trace_log"])).max() < 1e-8
    assert int((ref["accepted"] == 1).sum()) > 50


def test_density_only_chain_matches_segment_picture():
    """Density-density H_loc (KT_DENSITY_ONLY): the GPU chain (Krylov traces) against an
    oracle chain whose traces come from the segment picture (segment lengths and
    overlaps, oracle/segment.py), on the same uniforms: the same decisions and final
    configurations, the same trace and determinant weights."""
    from oracle.segment import SegmentTrace
    w = workloads.three_orbital()
    spec = w.model
    nw, steps = 16, 400
    P = Params(spec.n_orb, spec.U, spec.J, Up=spec.up, mu=spec.mu, delta=spec.delta, beta=spec.beta,
               trunc_eps=spec.trunc_eps, deg_tol=spec.deg_tol, density_only=True)
    om = Model(P)
    seg = SegmentTrace(spec.n_orb, spec.U, spec.J, spec.mu, spec.delta, spec.beta, Up=spec.up,
                       trunc_eps=spec.trunc_eps, deg_tol=spec.deg_tol)
    gm = engine.model_from_spec(spec, precision=kt.KT_FP64, flags=kt.KT_DENSITY_ONLY)
    assert kt.kt_model_query(gm)["n_kept"] == seg.n_kept
    table = workloads.semicircular_hybridization(spec.beta, 6, n_tau=2000)
    u = workloads.sweep_uniforms(steps, nw, seed=23)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=32, n_bins=20, measure_obs=False)
    sw.run(torch.as_tensor(u, device="cuda"), meas_every=8)
    ref = chain(om, Hyb(table, spec.beta), [[] for _ in range(nw)], u, k_cap=32, n_bins=20, meas_every=8,
                trace=seg)
    cnt = sw.counters()
    assert cnt["trace_errors"] == 0
    assert cnt["insert_accepted"] + cnt["remove_accepted"] == int((ref["accepted"] == 1).sum()) > 100
    cfg = sw.configs()
    for i in range(nw):
        assert cfg[i] == ref["configs"][i], i
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    assert (st["sign"] == ref["sign"]).all() and (st["trace_sign"] == ref["trace_sign"]).all()
    assert np.abs(st["trace_logabs"] - ref["trace_log"]).max() < 1e-9
    assert np.abs(st["det_logabs"] - (ref["logw"] - ref["trace_log"])).max() < 1e-8
    a = {k: v.cpu().numpy() for k, v in sw.accumulators().items()}
    assert np.allclose(a["order_sum"], ref["order_sum"])
    assert np.abs(a["g_tau"] - ref["g_acc"]).max() <= 1e-9 * max(1.0, np.abs(ref["g_acc"]).max())


def test_run_blocks_partition_the_accumulators():
    """run_blocks: the per-block sums add up to the running accumulators, the counters keep
    their totals, and the blocks feed a binning analysis of the double occupancy."""
    w = workloads.three_orbital()
    spec = w.model
    gm = engine.model_from_spec(spec, precision=kt.KT_FP32_KRYLOV)
    nw, steps, meas, nb = 64, 400, 10, 8
    table = workloads.semicircular_hybridization(spec.beta, 6, n_tau=2000)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=20, measure_obs=True)
    u = torch.as_tensor(workloads.sweep_uniforms(steps, nw, seed=41), device="cuda")
    blocks = sw.run_blocks(u, meas, nb)
    tot = sw.accumulators()
    for k in tot:
        s = sum(b[k] for b in blocks)
        assert torch.allclose(s, tot[k], rtol=1e-12, atol=1e-9), k
    cnt = sw.counters()
    assert cnt["measurements"] == steps // meas and cnt["insert_proposed"] + cnt["remove_proposed"] == nw * steps
    docc = np.stack([(b["obs_sum"][:, 6:9].mean(1) / b["sign_sum"]).cpu().numpy() for b in blocks], axis=1)
    r = engine.binning_analysis(docc)
    assert np.isfinite(r["error"]) and r["error"] > 0 and set(r["errors"]) >= {1, 2, 4}


def _thermal_five_orbital(nw, beta, seed):
    """Five-orbital configurations after 300 plain steps from Poisson(6) starts."""
    w = workloads.five_orbital()
    spec = workloads.five_orbital_sweep(beta).model
    gen = workloads.Workload(w.name, spec, start=w.start, order=w.order, lam=w.lam, cap=w.cap,
                             pattern_singles=w.pattern_singles)
    cand = workloads.generate_sequences(gen, 2 * nw, seed=seed)
    m = engine.model_from_spec(spec, precision=kt.KT_FP64)
    sg, _, _ = engine.trace(m, engine.DeviceSeqs.from_host(cand))
    ok = np.nonzero(sg.cpu().numpy() != 0)[0][:nw]
    table = workloads.semicircular_hybridization(beta, 10, n_tau=2000)
    sw = engine.Sweep(m, table, beta, nw, k_cap=128, n_bins=20)
    sw.set_configs(cand.subset(ok))
    sw.run(torch.as_tensor(workloads.sweep_uniforms(300, nw, seed=seed + 1), device="cuda"))
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    lens = st["lens"]
    seqs = workloads.Sequences(np.concatenate([[0], np.cumsum(lens)]).astype(np.int32),
                               np.concatenate([st["tau"][i, :lens[i]] for i in range(nw)]),
                               np.concatenate([st["flavor"][i, :lens[i]] for i in range(nw)]),
                               np.concatenate([st["dagger"][i, :lens[i]] for i in range(nw)]))
    return spec, table, seqs


@pytest.mark.parametrize("precision", [kt.KT_FP64, kt.KT_FP32_KRYLOV])
def test_cached_five_orbital_chains_match_uncached(precision):
    """Five orbitals at beta = 50 from thermalised configurations (about 160 operators):
    the cached chains take the decisions of the uncached ones on the same uniforms (FP64:
    every chain; FP32: the ratios differ by rounding, so a rare near-tie may flip) and
    track the same weights; the cached FP32 weights match the oracle's from scratch."""
    nw, steps, beta = 128, 300, 50.0
    spec, table, seqs = _thermal_five_orbital(nw, beta, seed=11)
    # not seed 12, the thermalisation's own stream (replaying it proposes exact time ties)
    u = torch.as_tensor(workloads.sweep_uniforms(steps, nw, seed=1011), device="cuda")
    gm = engine.model_from_spec(spec, precision=precision)
    runs = {}
    for c in (0, 512):
        sw = engine.Sweep(gm, table, beta, nw, k_cap=128, n_bins=20, cache_ops=c, measure_obs=True)
        sw.set_configs(seqs)
        sw.run(u, meas_every=10)
        runs[c] = (sw, {k: v.cpu().numpy() for k, v in sw.state().items()}, sw.counters())
    (a, sa, ca), (b, sb, cb) = runs[0], runs[512]
    # the beta/2 observables of the cached sweep come from its cached states
    oa, ob = a.accumulators()["obs_sum"].cpu().numpy(), b.accumulators()["obs_sum"].cpu().numpy()
    assert ca["trace_errors"] == 0 and cb["trace_errors"] == 0
    assert cb["insert_accepted"] + cb["remove_accepted"] > nw * steps // 10
    same = np.array([sa["lens"][i] == sb["lens"][i] and
                     np.array_equal(sa["tau"][i, :sa["lens"][i]], sb["tau"][i, :sb["lens"][i]]) for i in range(nw)])
    if precision == kt.KT_FP64:
        assert same.all()
        assert np.abs(sa["trace_logabs"] - sb["trace_logabs"]).max() < 1e-9
        assert np.abs(oa - ob).max() <= 1e-8 * max(1.0, np.abs(oa).max())
    else:
        # the two paths' FP32 ratios differ by rounding, far below any gap between log u5 and
        # log R that these uniforms produce: every chain takes the same decisions
        assert same.all()
        # the tracked traces are products of accepted FP32 ratios; after a refresh both sweeps
        # hold fresh evaluations of the same configurations, equal bit for bit and within RTOL
        # of the oracle
        da, db = a.refresh(), b.refresh()
        assert da["sign_mismatches"] == db["sign_mismatches"] == 0
        ra = {k: v.cpu().numpy() for k, v in a.state().items()}
        rb = {k: v.cpu().numpy() for k, v in b.state().items()}
        assert np.array_equal(ra["trace_logabs"], rb["trace_logabs"])
        om, _ = model_pair(spec, kt.KT_FP64)
        hyb = Hyb(table, beta)
        cfg = b.configs()
        for i in range(0, nw, 4):
            s_, lw, sT, lT = weight(om, hyb, cfg[i])
            assert s_ == rb["sign"][i] and sT == rb["trace_sign"][i], i
            assert abs(math.expm1(rb["trace_logabs"][i] - lT)) <= parity.RTOL[precision], i
        # the beta/2 observables of the two paths were taken on the same configurations
        assert np.abs(oa - ob).max() <= parity.RATIO_RTOL[precision] * max(1.0, np.abs(oa).max())


def test_cached_delayed_acceptance_matches_uncached():
    """Delayed acceptance with the cache: the same surrogate and uniforms give the same
    chain as without it (three orbitals, FP64)."""
    w = workloads.three_orbital()
    spec = w.model
    nw, steps = 64, 300
    gm = engine.model_from_spec(spec, precision=kt.KT_FP64)
    table = workloads.semicircular_hybridization(spec.beta, 6, n_tau=2000)
    u = torch.rand((steps, nw, 7), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    out = []
    for c in (0, 256):
        sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=10, cache_ops=c)
        net = engine.Surrogate(sw.n_features, max_batch=nw, seed=3)
        sw.set_surrogate(net)
        sw.run_da(u, meas_every=10)
        out.append((sw.configs(), sw.counters(), sw.state()["trace_logabs"].cpu().numpy()))
    assert out[0][0] == out[1][0]
    assert out[0][1] == out[1][1]
    assert out[0][1]["stage1_rejected"] > 0 and out[0][1]["insert_accepted"] > 0
    assert np.abs(out[0][2] - out[1][2]).max() < 1e-9


@pytest.mark.parametrize("precision", [kt.KT_FP64, kt.KT_FP32_KRYLOV])
def test_cached_sweep_long_run_weights_stay_exact(precision):
    """2,000 cached steps of 256 five-orbital chains at beta = 50 (thousands of accepted moves
    per chain's cache): the tracked trace of every chain equals a from-scratch evaluation of
    its final configuration (1e-9 FP64, RATIO_RTOL FP32), so the cache accumulates no error."""
    nw, beta = 256, 50.0
    spec, table, seqs = _thermal_five_orbital(nw, beta, seed=17)
    gm = engine.model_from_spec(spec, precision=precision)
    sw = engine.Sweep(gm, table, beta, nw, k_cap=128, n_bins=10, cache_ops=512)
    sw.set_configs(seqs)
    g = torch.Generator(device="cuda").manual_seed(19)
    for _ in range(4):
        sw.run(torch.rand((500, nw, 6), dtype=torch.float64, device="cuda", generator=g))
    cnt = sw.counters()
    assert cnt["trace_errors"] == 0 and cnt["insert_accepted"] + cnt["remove_accepted"] > 100 * nw
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    lens = st["lens"]
    final = workloads.Sequences(np.concatenate([[0], np.cumsum(lens)]).astype(np.int32),
                                np.concatenate([st["tau"][i, :lens[i]] for i in range(nw)]),
                                np.concatenate([st["flavor"][i, :lens[i]] for i in range(nw)]),
                                np.concatenate([st["dagger"][i, :lens[i]] for i in range(nw)]))
    s, l, stt = (t.cpu().numpy() for t in engine.trace(gm, engine.DeviceSeqs.from_host(final)))
    assert (stt == kt.KT_OK).all() and (s == st["trace_sign"]).all()
    tol = 1e-9 if precision == kt.KT_FP64 else parity.RATIO_RTOL[precision]
    assert np.abs(l - st["trace_logabs"]).max() <= tol, float(np.abs(l - st["trace_logabs"]).max())


def test_seven_orbital_cached_chains_match_uncached():
    """Seven orbitals (the 16-lane, 36-row cached kernel, writing states and measuring at beta/2
    from the cache): FP64 chains with and without the partial-state cache take the same
    decisions on the same uniforms and accumulate the same observables."""
    w = workloads.seven_orbital()
    spec = w.model
    gm = engine.model_from_spec(spec, precision=kt.KT_FP64)
    nw, steps = 16, 120
    table = workloads.semicircular_hybridization(spec.beta, 14, n_tau=2000, half_bandwidth=1.0)
    u = torch.as_tensor(workloads.sweep_uniforms(steps, nw, seed=9), device="cuda")
    out = []
    for c in (0, 256):
        sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=32, n_bins=10, measure_obs=True, cache_ops=c)
        sw.run(u, meas_every=10)
        out.append((sw.configs(), sw.counters(), {k: v.cpu().numpy() for k, v in sw.accumulators().items()},
                    sw.state()["trace_logabs"].cpu().numpy()))
    assert out[0][0] == out[1][0]
    assert out[0][1] == out[1][1] and out[0][1]["insert_accepted"] > 0 and out[0][1]["trace_errors"] == 0
    assert np.abs(out[0][3] - out[1][3]).max() < 1e-9
    oa, ob = out[0][2]["obs_sum"], out[1][2]["obs_sum"]
    # columns that the oracle leaves undefined beyond five orbitals are still computed on the GPU
    assert np.abs(oa - ob).max() <= 1e-8 * max(1.0, np.abs(oa).max())


def test_cached_sweep_restart_invalidates_the_cache():
    """set_configs in the middle of a cached run: the cache is invalidated and rebuilt from the
    new configurations, so the chains continue exactly as uncached ones do (FP64)."""
    w = workloads.three_orbital()
    spec = w.model
    gm = engine.model_from_spec(spec, precision=kt.KT_FP64)
    om = model_pair(spec, kt.KT_FP64)[0]
    table = workloads.semicircular_hybridization(spec.beta, 6, n_tau=2000)
    hyb = Hyb(table, spec.beta)
    cand = workloads.generate_sequences(w, 400, seed=19)
    keep = [i for i in range(cand.n)
            if max([sum(1 for t, f, d in zip(*[a.tolist() for a in cand.walker(i)]) if f == g and d == 1)
                    for g in range(6)] + [0]) <= 8
            and weight(om, hyb, list(zip(*[a.tolist() for a in cand.walker(i)])))[0] != 0][:16]
    assert len(keep) == 16
    restart = cand.subset(keep)
    u1 = torch.as_tensor(workloads.sweep_uniforms(120, 16, seed=20), device="cuda")
    u2 = torch.as_tensor(workloads.sweep_uniforms(120, 16, seed=21), device="cuda")
    out = []
    for c in (0, 128):
        sw = engine.Sweep(gm, table, spec.beta, 16, k_cap=16, n_bins=10, measure_obs=True, cache_ops=c)
        sw.run(u1, meas_every=10)
        sw.set_configs(restart)
        sw.run(u2, meas_every=10)
        out.append((sw.configs(), sw.counters(), sw.state()["trace_logabs"].cpu().numpy(),
                    sw.accumulators()["obs_sum"].cpu().numpy()))
    assert out[0][0] == out[1][0]
    assert out[0][1] == out[1][1]
    assert np.abs(out[0][2] - out[1][2]).max() < 1e-9
    assert np.abs(out[0][3] - out[1][3]).max() <= 1e-8 * max(1.0, np.abs(out[0][3]).max())


def test_memory_query_matches_the_allocation():
    """kt_sweep_memory_bytes against the device memory kt_sweep_create takes (free memory
    before and after, within the allocation granularity). A first small sweep loads the
    kernels, so the measured difference is the sweep's own allocations."""
    spec = workloads.five_orbital_sweep().model
    gm = engine.model_from_spec(spec, precision=kt.KT_FP32_KRYLOV)
    table = workloads.semicircular_hybridization(spec.beta, 10, n_tau=2000)
    warm = engine.Sweep(gm, table, spec.beta, 8, k_cap=8, n_bins=10, measure_obs=True, cache_ops=16)
    del warm
    nw = 512
    torch.cuda.synchronize()
    f0 = torch.cuda.mem_get_info()[0]
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=50, measure_obs=True, cache_ops=256)
    torch.cuda.synchronize()
    used = f0 - torch.cuda.mem_get_info()[0]
    want = kt.kt_sweep_memory_bytes(gm, nw, 64, 2000, 50, True, 256, 0)
    assert want > 100 * 2 ** 20
    assert abs(used - want) <= 8 * 2 ** 20 + 0.01 * want, (used, want)
    assert sw.n_walkers == nw
