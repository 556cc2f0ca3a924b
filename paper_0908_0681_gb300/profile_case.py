"""A small, fixed invocation of the engine for profiler captures.

    python -m paper_0908_0681_gb300.profile_case [--workload five_orbital] [--walkers 4096]
           [--precision fp32|fp64] [--launches 3] [--cached]

Builds the model, computes the current traces once (kt_trace) and then runs
`launches` trace-ratio calls (kt_trace_ratio) on rounds of moves with seeds
1000 + r. With --cached the ratios come from the partial-state cache of the same
configurations (kt_ratio_cache_build once, then kt_trace_ratio_cached). Everything
stays on the device; the process exits 0 on success.
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
    p.add_argument("--workload", default="five_orbital")
    p.add_argument("--walkers", type=int, default=4096)
    p.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    p.add_argument("--launches", type=int, default=3)
    p.add_argument("--flags", type=int, default=0)
    p.add_argument("--group-lanes", type=int, default=0, help="lanes per item (0: the model default)")
    p.add_argument("--cached", action="store_true", help="ratios from the partial-state cache")
    a = p.parse_args()
    import torch

    from paper_0908_0681_gb300 import engine, kt, workloads

    w = workloads.WORKLOADS[a.workload]()
    seqs = workloads.generate_sequences(w, a.walkers, seed=1)
    moves = [engine.DeviceMoves.from_host(workloads.generate_moves(w, seqs, seed=1000 + r)) for r in range(a.launches)]
    prec = kt.KT_FP32_KRYLOV if a.precision == "fp32" else kt.KT_FP64
    m = engine.model_from_spec(w.model, precision=prec, flags=a.flags)
    if a.group_lanes:
        kt.kt_model_set_tiling(m, a.group_lanes)
    d = engine.DeviceSeqs.from_host(seqs)
    ws = engine.workspace(m, seqs.n)
    cs, cl, st = engine.trace(m, d, ws=ws)
    cache = None
    if a.cached:
        cache = engine.RatioCache(m, seqs.n, max_ops=512)
        cache.build(d)
    for r in range(a.launches):
        if cache is not None:
            s, lr, st2 = cache.ratio(d, cs, cl, moves[r])
        else:
            s, lr, st2 = engine.trace_ratio(m, d, cs, cl, moves[r], ws=ws)
    torch.cuda.synchronize()
    bad = int((st != 0).sum().item()) + int((st2 != 0).sum().item())
    print(f"profile_case {a.workload} walkers={a.walkers} precision={a.precision} launches={a.launches} cached={a.cached} "
          f"info={kt.kt_model_query(m)} non_ok={bad}")
    return 0 if bad == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
