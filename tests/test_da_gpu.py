"""Learned delayed acceptance in the sweep (kt_sweep_collect, kt_sweep_run_da).

- The recorded training rows are the oracle's feature vectors of the same proposals
  (BF16-rounded, bit for bit) with their log trace ratios.
- With a constant surrogate (every weight zero, bias c: the prediction is exactly c on
  both sides) the two-stage chain takes the oracle's decisions step for step.
- A network trained on the chains' own ratios skips the trace of a large share of the
  proposals while the chains keep their statistics: the mean expansion order and G(tau)
  agree with plain Metropolis within 5 standard errors over independent chains.
- Multi-try delayed acceptance (kt_sweep_run_da_multi): with a constant surrogate the
  chains take the oracle's decisions try for try, and the tries-weighted accumulators equal
  the oracle's; on the five-orbital model with a trained surrogate the weighted statistics
  (order, G(tau), double occupancy, n_f) agree with plain Metropolis.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import mlp as ref  # noqa: E402
from oracle.ctqmc import Hyb, chain, chain_da_multi, propose, weight  # noqa: E402
from oracle.oracle import Model, Params  # noqa: E402
from paper_0908_0681_gb300 import engine, kt, workloads  # noqa: E402


def three_orbital(precision=kt.KT_FP64):
    spec = workloads.three_orbital().model
    P = Params(spec.n_orb, spec.U, spec.J, Up=spec.up, mu=spec.mu, delta=spec.delta, beta=spec.beta,
               trunc_eps=spec.trunc_eps, deg_tol=spec.deg_tol)
    table = workloads.semicircular_hybridization(spec.beta, 6, n_tau=2000)
    return spec, Model(P), engine.model_from_spec(spec, precision=precision), table


def bf16(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy()


def test_recorded_features_match_oracle():
    spec, om, gm, table = three_orbital()
    nw, steps = 4, 150
    u = workloads.sweep_uniforms(steps, nw, seed=44)
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=10)
    feats, targs = sw.collect(torch.as_tensor(u, device="cuda"), capacity=nw * steps)
    got = sorted(zip(targs.cpu().numpy().tolist(), [tuple(r) for r in feats.float().cpu().numpy().tolist()]))
    # the oracle's replay of the same plain chain
    hyb = Hyb(table, spec.beta)
    nf = 6
    cfg = [[] for _ in range(nw)]
    cur = [weight(om, hyb, c) for c in cfg]
    want = []
    for s in range(steps):
        for w in range(nw):
            mv = propose(cfg[w], u[s, w], nf, spec.beta, 64)
            if mv is None:
                continue
            new, lp, info = mv
            nwt = weight(om, hyb, new)
            if nwt[0] == 0:
                continue
            x = ref.features(cfg[w], nf, spec.beta, *info)
            lr_trace = nwt[3] - cur[w][3]
            want.append((float(np.float32(lr_trace if info[0] == 0 else -lr_trace)), tuple(bf16(x).tolist())))
            if (math.log(u[s, w, 5]) if u[s, w, 5] > 0 else -math.inf) < nwt[1] - cur[w][1] + lp:
                cfg[w], cur[w] = new, nwt
    want.sort()
    assert len(got) == len(want) > 100
    for (tg, fg), (tw, fw) in zip(got, want):
        assert fg == fw
        assert abs(tg - tw) <= 1e-6 * max(1.0, abs(tw))


def test_constant_surrogate_chain_matches_oracle():
    spec, om, gm, table = three_orbital()
    nw, steps, c = 16, 300, -0.3
    n_in = ref.n_inputs(6)
    p = {k: np.zeros(s) for k, s in ref.shapes(n_in).items()}
    p["b3"] = np.array([c])
    net = engine.Surrogate(n_in, max_batch=nw, params=ref.pack(p))
    u = np.random.default_rng(55).random((steps, nw, 7))
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=10)
    sw.set_surrogate(net)
    sw.run_da(torch.as_tensor(u, device="cuda"))
    cf = float(np.float32(c))
    # the network's constant output c is the insertion prediction; a removal gets -c
    out = chain(om, Hyb(table, spec.beta), [[] for _ in range(nw)], u, k_cap=64,
                surrogate=lambda ops, kind, *a: cf if kind == 0 else -cf)
    cnt = sw.counters()
    assert sw.configs() == out["configs"]
    assert cnt["stage1_rejected"] == int((out["accepted"] == -2).sum()) > 0
    assert cnt["insert_accepted"] + cnt["remove_accepted"] == int((out["accepted"] == 1).sum())


def test_trained_surrogate_saves_traces_and_keeps_statistics():
    spec, om, gm, table = three_orbital(kt.KT_FP32_KRYLOV)
    nw, nb = 1024, 10
    g = torch.Generator(device="cuda").manual_seed(9)

    def uni(n, k):
        return torch.rand((n, nw, k), dtype=torch.float64, device="cuda", generator=g)

    # training data from the chains themselves
    base = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=nb)
    base.run(uni(400, 6))
    X, t = base.collect(uni(300, 6), capacity=400_000)
    net = engine.Surrogate(base.n_features, max_batch=4096, seed=1)
    hist = net.train(X, t.clamp(-25.0, 10.0), epochs=4, batch=4096, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    # equal numbers of proposals, plain and delayed, from the same thermalised start
    res = {}
    for mode in ("plain", "da"):
        sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=nb)
        sw.run(uni(400, 6))
        sw.reset_accumulators()
        if mode == "plain":
            sw.run(uni(1500, 6), meas_every=10)
        else:
            sw.set_surrogate(net)
            sw.run_da(uni(1500, 7), meas_every=10)
        a = {k: v.cpu().numpy() for k, v in sw.accumulators().items()}
        res[mode] = (a, sw.counters())
    (ap, cp), (ad, cd) = res["plain"], res["da"]
    assert cd["trace_evaluations"] < 0.7 * cp["trace_evaluations"], (cd, cp)

    def per_walker(a):
        order = a["order_sum"].sum(1) / a["sign_sum"]
        gt = (a["g_tau"] * (nb / spec.beta ** 2) / a["sign_sum"][:, None, None]).mean(1)
        return order, gt

    op, gp = per_walker(ap)
    od, gd = per_walker(ad)
    se = math.sqrt(op.var(ddof=1) / nw + od.var(ddof=1) / nw)
    assert abs(op.mean() - od.mean()) < 5 * se, (op.mean(), od.mean(), se)
    seg = np.sqrt(gp.var(0, ddof=1) / nw + gd.var(0, ddof=1) / nw)
    assert np.all(np.abs(gp.mean(0) - gd.mean(0)) < 5 * seg + 1e-4)


def test_multi_try_constant_surrogate_matches_oracle():
    spec, om, gm, table = three_orbital()
    nw, steps, T, c, nb = 16, 240, 4, -0.3, 10
    n_in = ref.n_inputs(6)
    p = {k: np.zeros(s) for k, s in ref.shapes(n_in).items()}
    p["b3"] = np.array([c])
    net = engine.Surrogate(n_in, max_batch=nw * T, params=ref.pack(p))
    u = np.random.default_rng(56).random((steps, nw, T, 7))
    sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=nb, measure_obs=True)
    sw.set_surrogate(net)
    sw.run_da_multi(torch.as_tensor(u, device="cuda"), meas_every=6)
    cf = float(np.float32(c))
    out = chain_da_multi(om, Hyb(table, spec.beta), [[] for _ in range(nw)], u,
                         lambda ops, kind, *a: cf if kind == 0 else -cf, k_cap=64, n_bins=nb, meas_every=6,
                         observables=True)
    cnt = sw.counters()
    assert sw.configs() == out["configs"]
    k = out["counts"]
    assert cnt["insert_proposed"] == k["insertions"] and cnt["remove_proposed"] == k["removals"]
    assert cnt["null_moves"] == k["null"]
    assert cnt["stage1_rejected"] == k["stage1_rejected"] > 0
    assert cnt["insert_accepted"] + cnt["remove_accepted"] == int((out["accepted"] == 1).sum())
    assert cnt["trace_evaluations"] == int((out["accepted"] != -2).sum())
    assert out["tries"].mean() > 1.2
    a = {key: v.cpu().numpy() for key, v in sw.accumulators().items()}
    assert np.allclose(a["sign_sum"], out["sign_sum"]) and np.abs(a["sign_sum"]).sum() > nw
    assert np.allclose(a["order_sum"], out["order_sum"])
    assert np.abs(a["g_tau"] - out["g_acc"]).max() <= 1e-9 * max(1.0, np.abs(out["g_acc"]).max())
    assert np.abs(a["obs_sum"] - out["obs_sum"]).max() <= 1e-8 * max(1.0, np.abs(out["obs_sum"]).max())


def test_multi_try_five_orbital_statistics():
    """Five-orbital model, beta 50, FP32-Krylov traces, 1,024 chains from Poisson(6) starting
    configurations thermalised by 2,000 plain steps; from that state, plain Metropolis
    (1,600 steps, measured every 10) and four-try delayed acceptance (800 call steps,
    measured every 5): per-chain estimates of the order, G(tau) and every beta/2 observable
    (n_f, double occupancies, sector probabilities) agree within 5 standard errors, and the
    delayed chains evaluate fewer traces per Metropolis step."""
    w = workloads.five_orbital()
    spec = workloads.five_orbital_sweep().model
    gen = workloads.Workload(w.name, spec, start=w.start, order=w.order, lam=w.lam, cap=w.cap,
                             pattern_singles=w.pattern_singles)
    gm = engine.model_from_spec(spec, precision=kt.KT_FP32_KRYLOV)
    table = workloads.semicircular_hybridization(spec.beta, 10, n_tau=2000)
    nw, nb, T = 1024, 10, 4
    g = torch.Generator(device="cuda").manual_seed(19)

    def uni(*shape):
        return torch.rand(shape, dtype=torch.float64, device="cuda", generator=g)

    cand = workloads.generate_sequences(gen, 2 * nw, seed=23)
    sg, _, _ = engine.trace(gm, engine.DeviceSeqs.from_host(cand))
    ok = np.nonzero(sg.cpu().numpy() != 0)[0][:nw]
    assert len(ok) == nw
    base = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=nb)
    base.set_configs(cand.subset(ok))
    base.run(uni(2000, nw, 6))
    st = {k: v.cpu().numpy() for k, v in base.state().items()}
    L = st["lens"]
    thermal = workloads.Sequences(np.concatenate([[0], np.cumsum(L)]).astype(np.int32),
                                  np.concatenate([st["tau"][i, :L[i]] for i in range(nw)]),
                                  np.concatenate([st["flavor"][i, :L[i]] for i in range(nw)]),
                                  np.concatenate([st["dagger"][i, :L[i]] for i in range(nw)]))
    X, t = base.collect(uni(300, nw, 6), capacity=400_000)
    net = engine.Surrogate(base.n_features, max_batch=nw * T, seed=2)
    hist = net.train(X, t.clamp(-25.0, 10.0), epochs=6, batch=4096, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    res = {}
    for mode in ("plain", "multi"):
        sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=nb, measure_obs=True)
        sw.set_configs(thermal)
        if mode == "plain":
            sw.run(uni(1600, nw, 6), meas_every=10)
        else:
            sw.set_surrogate(net)
            sw.run_da_multi(uni(800, nw, T, 7), meas_every=5)
        a = {k: v.cpu().numpy() for k, v in sw.accumulators().items()}
        res[mode] = (a, sw.counters())
    (ap, cp), (am, cm) = res["plain"], res["multi"]
    steps_m = cm["insert_proposed"] + cm["remove_proposed"]
    assert steps_m > 1.5 * 800 * nw
    assert cm["trace_evaluations"] / steps_m < 0.5 * cp["trace_evaluations"] / (1600 * nw)

    def per_chain(a):
        # per-chain weighted means: order, G(tau) averaged over flavors, and every beta/2
        # observable (n_f, double occupancies, sector probabilities)
        s = a["sign_sum"]
        order = a["order_sum"].sum(1) / s
        gt = (a["g_tau"] * (nb / spec.beta ** 2) / s[:, None, None]).mean(1)
        return order, gt, a["obs_sum"] / s[:, None]

    op, gp, obp = per_chain(ap)
    om_, gm_, obm = per_chain(am)
    se = math.sqrt(op.var(ddof=1) / nw + om_.var(ddof=1) / nw)
    assert abs(op.mean() - om_.mean()) < 5 * se, (op.mean(), om_.mean(), se)
    seg = np.sqrt(gp.var(0, ddof=1) / nw + gm_.var(0, ddof=1) / nw)
    assert np.all(np.abs(gp.mean(0) - gm_.mean(0)) < 5 * seg + 1e-4)
    seo = np.sqrt(obp.var(0, ddof=1) / nw + obm.var(0, ddof=1) / nw)
    assert np.all(np.abs(obp.mean(0) - obm.mean(0)) < 5 * seo + 1e-6), (obp.mean(0), obm.mean(0), seo)


def test_multi_try_features_equal_single_try_features():
    """The multi-try path builds its features per walker from a shared next-same-flavor table;
    with one try and a network whose prediction depends on every feature (random weights), it
    takes exactly the decisions of kt_sweep_run_da, whose features come from the per-proposal
    kernel (the values are the same up to the order of floating-point additions)."""
    spec, om, gm, table = three_orbital()
    nw, steps = 64, 300
    net = engine.Surrogate(ref.n_inputs(6), max_batch=nw, seed=5)
    u = np.random.default_rng(57).random((steps, nw, 7))
    res = []
    for multi in (False, True):
        sw = engine.Sweep(gm, table, spec.beta, nw, k_cap=64, n_bins=10)
        sw.set_surrogate(net)
        if multi:
            sw.run_da_multi(torch.as_tensor(u[:, :, None, :].copy(), device="cuda"))
        else:
            sw.run_da(torch.as_tensor(u, device="cuda"))
        res.append((sw.configs(), sw.counters()))
    (ca, ka), (cb, kb) = res
    assert ka["stage1_rejected"] > 0.1 * nw * steps
    assert ca == cb
    for k in ("insert_proposed", "remove_proposed", "insert_accepted", "remove_accepted", "stage1_rejected",
              "trace_evaluations", "null_moves"):
        assert ka[k] == kb[k], k
