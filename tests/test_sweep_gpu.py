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


def model_pair(spec, precision):
    P = Params(spec.n_orb, spec.U, spec.J, Up=spec.up, mu=spec.mu, delta=spec.delta, beta=spec.beta,
               trunc_eps=spec.trunc_eps, deg_tol=spec.deg_tol)
    return Model(P), engine.model_from_spec(spec, precision=precision)


def run_both(spec, nw, steps, k_cap, n_bins, meas_every, seed, precision=kt.KT_FP64, observables=True):
    om, gm = model_pair(spec, precision)
    table = workloads.semicircular_hybridization(spec.beta, 2 * spec.n_orb, n_tau=2000)
    u = workloads.sweep_uniforms(steps, nw, seed=seed)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=k_cap, n_bins=n_bins, measure_obs=observables)
    sw.run(torch.as_tensor(u, device="cuda"), meas_every=meas_every)
    ref = chain(om, Hyb(table, spec.beta), [[] for _ in range(nw)], u, k_cap=k_cap, n_bins=n_bins,
                meas_every=meas_every, observables=observables)
    return om, Hyb(table, spec.beta), sw, ref


@pytest.mark.parametrize("k_cap", [64, 2])
def test_three_orbital_chain_matches_oracle(k_cap):
    w = workloads.three_orbital()
    spec = w.model
    nw, steps = 16, 400
    om, hyb, sw, ref = run_both(spec, nw, steps, k_cap, n_bins=20, meas_every=8, seed=21)
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


def test_seven_orbital_fp32_chain_weights():
    """Seven orbitals (36-row kernel blocks, N_tr = 63): chains of FP32-Krylov trace ratios
    with the semicircular bath of bandwidth 2 keep weights consistent with the oracle."""
    w = workloads.seven_orbital()
    spec = w.model
    om, gm = model_pair(spec, kt.KT_FP32_KRYLOV)
    nw, steps = 32, 200
    table = workloads.semicircular_hybridization(spec.beta, 14, n_tau=2000, half_bandwidth=1.0)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=32, n_bins=10)
    sw.run(torch.as_tensor(workloads.sweep_uniforms(steps, nw, seed=7), device="cuda"))
    cnt = sw.counters()
    assert cnt["trace_errors"] == 0 and cnt["insert_accepted"] > 0
    st = {k: v.cpu().numpy() for k, v in sw.state().items()}
    hyb = Hyb(table, spec.beta)
    for i, ops in enumerate(sw.configs()):
        s, lw, sT, lT = weight(om, hyb, ops)
        assert s == st["sign"][i] and sT == st["trace_sign"][i], i
        assert abs(math.expm1(st["trace_logabs"][i] - lT)) < 5e-5, i   # the FP32 ratio bound at seven orbitals
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
