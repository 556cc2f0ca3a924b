"""Comparison rules between the CUDA path and the oracle (used by the GPU tests).

Conditioning classes (from the FP64 oracle and its long-double twin):
  0 structural zero - the oracle's value is exactly zero: the GPU sign must be 0;
  1 numerical zero  - FP64 and long double disagree beyond 1e-8 relative: the exact
                      value is zero by a symmetry that the (n_up, n_dn) sectors do not
                      resolve; the GPU may return 0 or a value with
                      |T~| <= zero_tol * N_tr;
  2 regular         - signs equal and |T_gpu / T_ext - 1| <= rtol.
rtol = 1e-10 for the FP64 path and 1e-5 for the FP32-Krylov path; zero_tol =
1e-12 and 1e-6 respectively. The reference value is the long-double twin,
because the FP64 oracle's own rounding reaches ~5e-11 relative on the
5-orbital workload.
"""
from __future__ import annotations

import math

import numpy as np

from oracle.oracle import Model, Params, SeqBatch, classify, ratio

RTOL = {0: 1e-10, 1: 1e-5}       # keyed by precision (KT_FP64 = 0, KT_FP32_KRYLOV = 1)
ZERO_TOL = {0: 1e-12, 1: 1e-6}
# A ratio formed end to end from two of the path's own traces, T_new / T_cur, each within
# RTOL of the exact value: |(1 + e1) / (1 + e2) - 1| <= (e1 + e2) / (1 - e2) <= 2 RTOL (1 + RTOL).
# Ratios against the oracle's current trace carry only the new trace's error and use RTOL.
RATIO_RTOL = {k: 2.0 * v * (1.0 + v) for k, v in RTOL.items()}


def oracle_pair(spec, trunc_eps=None, density_only=False):
    P = Params(spec.n_orb, spec.U, spec.J, Up=spec.up, mu=spec.mu, delta=spec.delta, beta=spec.beta,
               trunc_eps=spec.trunc_eps if trunc_eps is None else trunc_eps, deg_tol=spec.deg_tol,
               density_only=density_only)
    return Model(P), Model(P, "ext")


def seqbatch(seqs) -> SeqBatch:
    return SeqBatch(seqs.offsets, seqs.tau, seqs.flavor, seqs.dagger)


def oracle_traces(o64, ox, seqs):
    sb = seqbatch(seqs)
    s64, l64, _ = o64.trace(sb)
    sx, lx, _ = ox.trace(sb)
    return classify(s64, l64, sx, lx), sx, lx


def oracle_ratios(o64, ox, seqs, cur_sign, cur_logabs, moves):
    sb = seqbatch(seqs)
    _, _, ns64, nl64 = ratio(o64, sb, cur_sign, cur_logabs, moves.as_dict())
    _, _, nsx, nlx = ratio(ox, sb, cur_sign, cur_logabs, moves.as_dict())
    return classify(ns64, nl64, nsx, nlx), nsx, nlx


def compare(cls, ref_sign, ref_log, gpu_sign, gpu_log, precision, n_tr, beta_e0, label=""):
    """Check every element; returns a dict of counts and the worst relative error."""
    rtol, ztol = RTOL[precision], ZERO_TOL[precision]
    beta_e0 = np.broadcast_to(np.asarray(beta_e0, dtype=np.float64), (len(cls),))
    worst = 0.0
    bad = []
    for i in range(len(cls)):
        c = int(cls[i])
        if c == 0:
            if gpu_sign[i] != 0:
                bad.append((i, "structural zero expected", int(gpu_sign[i]), float(gpu_log[i])))
        elif c == 1:
            if gpu_sign[i] != 0:
                lt = float(gpu_log[i]) + float(beta_e0[i])   # log|T~| of the GPU value
                if not (lt <= math.log(ztol * n_tr)):
                    bad.append((i, "numerical zero too large", lt))
        else:
            if gpu_sign[i] != ref_sign[i]:
                bad.append((i, "sign", int(gpu_sign[i]), int(ref_sign[i])))
                continue
            e = abs(math.expm1(float(gpu_log[i]) - float(ref_log[i])))
            worst = max(worst, e)
            if not (e <= rtol):
                bad.append((i, "relative error", e, float(gpu_log[i]), float(ref_log[i])))
    assert not bad, f"{label}: {len(bad)} mismatches, first {bad[:5]}"
    return {"structural": int((cls == 0).sum()), "numerical": int((cls == 1).sum()),
            "regular": int((cls == 2).sum()), "max_rel_err": worst}
