"""A fixed invocation of the CT-HYB sweep for profiler captures.

    python -m paper_0908_0681_gb300.profile_sweep [--beta 50] [--chains 1024] [--steps 20]
           [--therm 200] [--collect 100] [--mode plain|da|both|multi] [--tries 8] [--cache-ops 0]
           [--precision fp32|fp64] [--k-cap 128]

Five-orbital model with the semicircular bath (2,000 tau points); the chains start from
Poisson(6) configurations (kt_sweep_set_configs) and thermalise `therm` steps. For
`da` and `multi`, a surrogate is trained for one epoch on `collect` steps of the chains' own
ratios. Then `steps` plain and/or delayed-acceptance steps (`multi`: call steps of up to
`tries` stage-1 tries, kt_sweep_run_da_multi) run, measuring every 10 steps, with
the partial-state cache when --cache-ops > 0. Prints the CUDA-event time per step and
the trace pipeline's work per proposal. Exits 0 when no chain reported a trace error.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--beta", type=float, default=50.0)
    p.add_argument("--chains", type=int, default=1024)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--therm", type=int, default=200)
    p.add_argument("--mode", choices=["plain", "da", "both", "multi"], default="both")
    p.add_argument("--tries", type=int, default=8, help="stage-1 tries per call step of --mode multi")
    p.add_argument("--collect", type=int, default=100, help="steps of training data for the surrogate")
    p.add_argument("--cache-ops", type=int, default=0)
    p.add_argument("--k-cap", type=int, default=128)
    p.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    a = p.parse_args()
    import numpy as np
    import torch

    from paper_0908_0681_gb300 import engine, kt, workloads

    nw = a.chains
    w = workloads.five_orbital()
    spec = workloads.five_orbital_sweep(a.beta).model
    gen = workloads.Workload(w.name, spec, start=w.start, order=w.order, lam=w.lam, cap=w.cap,
                             pattern_singles=w.pattern_singles)
    cand = workloads.generate_sequences(gen, 2 * nw, seed=7)
    model = engine.model_from_spec(spec, precision=kt.KT_FP32_KRYLOV if a.precision == "fp32" else kt.KT_FP64)
    sg, _, _ = engine.trace(model, engine.DeviceSeqs.from_host(cand))
    ok = np.nonzero(sg.cpu().numpy() != 0)[0][:nw]
    table = workloads.semicircular_hybridization(a.beta, 2 * spec.n_orb, n_tau=2000)
    sw = engine.Sweep(model, table, a.beta, nw, k_cap=a.k_cap, n_bins=200, measure_obs=True, cache_ops=a.cache_ops)
    sw.set_configs(cand.subset(ok))
    g = torch.Generator(device="cuda").manual_seed(3)

    def uni(n, k):
        return torch.rand((n, nw, k), dtype=torch.float64, device="cuda", generator=g)

    sw.run(uni(a.therm, 6))

    def timed(fn, u):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c0 = sw.counters()
        fn(u, meas_every=10)
        e1.record()
        torch.cuda.synchronize()
        c1 = sw.counters()
        ms = e0.elapsed_time(e1) / u.shape[0]
        mh = (c1["insert_proposed"] + c1["remove_proposed"] - c0["insert_proposed"] - c0["remove_proposed"]) / u.shape[0]
        st = engine.new_stats()
        sw.set_stats(st)
        fn(u[:10])
        sw.set_stats(None)
        w = kt.stats_from_tensor(st)
        per = {k: round(w[k] / (10 * nw), 3) for k in ("intervals", "ops_applied", "krylov_iters", "items_alive")}
        print(f"  {fn.__name__}: {ms:.3f} ms per call step, {mh / ms * 1e3:.0f} Metropolis steps/s, "
              f"work per chain and call step {per}")

    if a.mode in ("plain", "both"):
        timed(sw.run, uni(a.steps, 6))
    if a.mode in ("da", "both"):
        X, t = sw.collect(uni(a.collect, 6), capacity=a.collect * nw)
        net = engine.Surrogate(sw.n_features, max_batch=max(4096, nw), seed=1)
        net.train(X, t.clamp(-25.0, 10.0), epochs=1, batch=4096, lr=3e-3)
        sw.set_surrogate(net)
        timed(sw.run_da, uni(a.steps, 7))
    if a.mode == "multi":
        X, t = sw.collect(uni(a.collect, 6), capacity=a.collect * nw)
        net = engine.Surrogate(sw.n_features, max_batch=max(4096, a.tries * nw), seed=1)
        net.train(X, t.clamp(-25.0, 10.0), epochs=1, batch=4096, lr=3e-3)
        sw.set_surrogate(net)
        u = torch.rand((a.steps, nw, a.tries, 7), dtype=torch.float64, device="cuda", generator=g)
        timed(sw.run_da_multi, u)
    torch.cuda.synchronize()
    c = sw.counters()
    print(f"profile_sweep beta={a.beta:g} chains={nw} steps={a.steps} mode={a.mode} cache_ops={a.cache_ops} "
          f"precision={a.precision} counters={c}")
    return 0 if c["trace_errors"] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
