"""Plain CT-HYB Markov chain of the hybridization expansion (test infrastructure only).

Only the tests and the smoke check import this module; the product library never
calls it. Every weight is computed from scratch from its
definition; nothing is updated incrementally.

Weight of a configuration (Sec. II, Eq. (weight_strong) with a hybridization that is
diagonal in the flavors). A configuration is a time-ordered list of c_f^+ / c_f
operators; for each flavor f let tau'_1 < ... < tau'_k be the creator times and
tau_1 < ... < tau_k the annihilator times. Then

    w(c) = s_P(c) * T(c) * prod_f det G_f,      G_f[i, j] = Fh_f(tau'_i - tau_j)

  T      the truncated local trace of the operator sequence (oracle.Model.trace);
  Fh_f   Fh(x) = F_f(x) for x >= 0 and -F_f(x + beta) for x < 0, where
         F_f(tau) = sum_p |V_p|^2 e^{-tau eps_p} / (1 + e^{-beta eps_p}) = -Delta_f(tau)
         is the bath correlator <T a_p(tau) a_p^+(0)> summed with the hybridization
         amplitudes (positive on [0, beta]), tabulated on n_tau + 1 equidistant
         points and interpolated linearly;
  s_P    the sign of the permutation that takes the bath operators, written flavor
         by flavor as a(tau'_1) a^+(tau_1) a(tau'_2) a^+(tau_2) ..., into descending
         time order (Wick's theorem for the bath, whose operators sit at the times
         of the impurity operators they pair with).

Reading of the expansion (the paper gives the structure of Eq. (weight_strong) but
no sign convention): the hybridization term V c^+ a + V* a^+ c puts a bath a at
every c^+ time and a bath a^+ at every c time; moving the bath operators past the
impurity operators inside the time-ordered product of these even bilinears gives
no sign, so the impurity trace keeps the plain time order of the operator
sequence and the bath factor is the time-ordered product of the bath operators.

Markov chain (Sec. II: "random insertion or removal of pairs of creation and
annihilation operators"; the proposal probabilities are the usual ones of the
segment/anti-segment scheme of the hybridization expansion). Per step and walker six
uniforms u[0..5] in [0, 1):
  u0 < 1/2 insert, else remove; flavor f = floor(u1 * n_flavors).
  insert: t1 = u2 beta. With no f operators: a coin u4 < 1/2 picks a segment (c^+ at
      t1, c at t2) or an anti-segment (c at t1, c^+ at t2), l = beta. Otherwise the
      next f operator after t1 (cyclically) decides: a c^+ next means t1 is empty, so
      a segment; a c next, an anti-segment; l is the distance to it. t2 = t1 + u3 l
      (mod beta). Proposal factor: beta^2 for k_f = 0, else beta l / (2 (k_f + 1)).
  remove: with k_f pairs, the j = floor(u2 * 2 k_f)-th f operator in time order goes
      with the next f operator after it (cyclically). Proposal factor: 1 / beta^2 for
      k_f = 1, else 2 k_f / (beta l'), l' the distance from the first removed
      operator to the f operator that follows the pair.
  accept when log(u5) < log|w_new / w_old| + log(proposal factor).
  Null moves (no change, no acceptance test): removing from an empty flavor,
  inserting beyond k_cap pairs, t1 >= beta after rounding, or t2 == t1.
Delayed acceptance (Christen & Fox 2005) with a surrogate r~ of log|T_new / T_old|: a
seventh uniform u6 per step; stage 1 accepts when
  log(u6) < r~ + log|bath factor ratio| + log(proposal factor),
and only then is the trace evaluated; stage 2 accepts when log(u5) < log|T_new/T_old| - r~.
This second stage is the Christen-Fox one, min(1, R alpha1(y, x) / alpha1(x, y)), for a
surrogate that is antisymmetric (the reverse move gets -r~): the chain then satisfies
detailed balance with respect to w. The surrogate callable must have that property.
Measurements every meas_every steps, weighted by the sign of w:
  G_f(tau) = (1/beta) < sum_{ij} M_ji dh(tau, tau_j - tau'_i) >,  M = G_f^{-1},
  dh(tau, x) = delta(tau - x) for x > 0 and -delta(tau - x - beta) for x < 0,
  accumulated in n_bins bins of [0, beta); the expansion order of every flavor; and
  the observables of oracle.measure at beta/2.
"""
from __future__ import annotations

import math

import numpy as np

from oracle.oracle import Model, SeqBatch, measure


class Hyb:
    """F_f(tau) on tau_i = i beta / n_tau, i = 0 .. n_tau, for every flavor."""

    def __init__(self, table: np.ndarray, beta: float):
        self.table = np.asarray(table, dtype=np.float64)
        self.beta = float(beta)
        self.n_tau = self.table.shape[1] - 1

    def F(self, f: int, tau: float) -> float:
        pos = tau / self.beta * self.n_tau
        i = int(math.floor(pos))
        i = min(max(i, 0), self.n_tau - 1)
        fr = pos - i
        a, b = self.table[f, i], self.table[f, i + 1]
        return a + fr * (b - a)

    def Fh(self, f: int, x: float) -> float:
        return self.F(f, x) if x >= 0.0 else -self.F(f, x + self.beta)


def flavor_times(ops, f):
    cre = sorted(t for t, g, d in ops if g == f and d == 1)
    ann = sorted(t for t, g, d in ops if g == f and d == 0)
    return cre, ann


def bath_matrix(hyb: Hyb, f: int, cre, ann) -> np.ndarray:
    return np.array([[hyb.Fh(f, tc - ta) for ta in ann] for tc in cre], dtype=np.float64).reshape(len(cre), len(ann))


def permutation_sign(ops, nf) -> int:
    """s_P: sign of sorting the bath operators, written flavor by flavor as
    a(tau'_1) a^+(tau_1) a(tau'_2) a^+(tau_2) ..., into descending time order."""
    seq = []
    for f in range(nf):
        cre, ann = flavor_times(ops, f)
        for tc, ta in zip(cre, ann):
            seq += [tc, ta]
    inv = 0
    for a in range(len(seq)):
        for b in range(a + 1, len(seq)):
            if seq[a] < seq[b]:
                inv += 1
    return -1 if inv % 2 else 1


def bath_weight(hyb: Hyb, ops, nf: int):
    """(sign, log|.|) of s_P * prod_f det G_f alone (no trace); sign 0 when singular."""
    sgn, lw = permutation_sign(ops, nf), 0.0
    for f in range(nf):
        cre, ann = flavor_times(ops, f)
        if len(cre) != len(ann):
            return 0, -math.inf
        if not cre:
            continue
        s, ld = np.linalg.slogdet(bath_matrix(hyb, f, cre, ann))
        if s == 0:
            return 0, -math.inf
        sgn *= int(s)
        lw += float(ld)
    return sgn, lw


def weight(model: Model, hyb: Hyb, ops, trace=None):
    """(sign, log|w|, sign_T, log|T|) of a configuration; sign 0 when w = 0. `trace`, when
    given, is a callable ops -> (sign, log|T|) that replaces model.trace (the segment
    picture of oracle/segment.py for the density-density model)."""
    nf = 2 * model.p.n_orb
    for f in range(nf):
        cre, ann = flavor_times(ops, f)
        if len(cre) != len(ann):
            return 0, -math.inf, 0, -math.inf
    if trace is None:
        sT, lT, _ = model.trace(SeqBatch.from_lists([ops]))
        sT, lT = int(sT[0]), float(lT[0])
    else:
        sT, lT = trace(ops)
    if sT == 0:
        return 0, -math.inf, 0, -math.inf
    sgn, logw = sT * permutation_sign(ops, nf), lT
    for f in range(nf):
        cre, ann = flavor_times(ops, f)
        if not cre:
            continue
        s, ld = np.linalg.slogdet(bath_matrix(hyb, f, cre, ann))
        if s == 0:
            return 0, -math.inf, sT, lT
        sgn *= int(s)
        logw += float(ld)
    return sgn, logw, sT, lT


def _insert(ops, t, f, d):
    pos = 0
    while pos < len(ops) and ops[pos][0] <= t:
        pos += 1
    return ops[:pos] + [(t, f, d)] + ops[pos:]


def propose(ops, u, nf, beta, k_cap):
    """The move of one step: (new ops, log proposal factor, (kind, flavor, t_first,
    t_second, first operator is a c^+)), or None for a null move."""
    f = min(int(u[1] * nf), nf - 1)
    fidx = [i for i, (t, g, d) in enumerate(ops) if g == f]
    k = len(fidx) // 2
    if u[0] < 0.5:
        if k >= k_cap:
            return None
        t1 = u[2] * beta
        if not t1 < beta:
            return None
        if k == 0:
            seg = u[4] < 0.5
            lmax = beta
        else:
            nxt = [i for i in fidx if ops[i][0] > t1]
            j = nxt[0] if nxt else fidx[0]
            seg = ops[j][2] == 1
            tn = ops[j][0]
            lmax = tn - t1 if tn > t1 else tn + beta - t1
        t2 = t1 + u[3] * lmax
        if t2 >= beta:
            t2 -= beta
        if t2 == t1:
            return None
        td, ta = (t1, t2) if seg else (t2, t1)
        new = ops
        first, second = ((td, 1), (ta, 0)) if td < ta else ((ta, 0), (td, 1))
        new = _insert(new, first[0], f, first[1])
        new = _insert(new, second[0], f, second[1])
        lp = 2.0 * math.log(beta) if k == 0 else math.log(beta * lmax / (2.0 * (k + 1)))
        return new, lp, (0, f, t1, t2, bool(seg))
    if k == 0:
        return None
    j = min(int(u[2] * 2 * k), 2 * k - 1)
    a = fidx[j]
    b = fidx[(j + 1) % (2 * k)]
    t1 = ops[a][0]
    if k == 1:
        lp = -2.0 * math.log(beta)
    else:
        c = fidx[(j + 2) % (2 * k)]
        tc = ops[c][0]
        lmax = tc - t1 if tc > t1 else tc + beta - t1
        lp = math.log(2.0 * k / (beta * lmax))
    new = [op for i, op in enumerate(ops) if i not in (a, b)]
    return new, lp, (1, f, t1, ops[b][0], ops[a][2] == 1)


def chain(model: Model, hyb: Hyb, init, uniforms: np.ndarray, k_cap: int = 64, n_bins: int = 50,
          meas_every: int = 0, observables: bool = False, surrogate=None, trace=None):
    """Run every walker's chain with the given uniforms [n_steps, n_walkers, 6] (7 with a
    surrogate: a callable (ops, kind, flavor, t_first, t_second, seg) -> predicted
    log|T_new / T_old|, used for delayed acceptance). `trace` replaces model.trace in every
    weight (see weight()).

    Returns a dict: accepted [n_steps, n_walkers] (1 accepted, 0 rejected, -1 null,
    -2 rejected at stage 1),
    configs (final op lists), sign / logw (final weights, recomputed), and when
    meas_every > 0: g_acc [n_walkers, nf, n_bins], sign_sum, order_sum [n_walkers, nf],
    n_meas, and obs_sum [n_walkers, nobs] if observables.
    """
    beta = model.p.beta
    nf = 2 * model.p.n_orb
    n_steps, nw, _ = uniforms.shape
    configs = [list(c) for c in init]
    cur = [weight(model, hyb, c, trace) for c in configs]
    acc = np.zeros((n_steps, nw), dtype=np.int8)
    g_acc = np.zeros((nw, nf, n_bins))
    sign_sum = np.zeros(nw)
    order_sum = np.zeros((nw, nf))
    obs_sum = None
    n_meas = 0
    for step in range(n_steps):
        for w in range(nw):
            mv = propose(configs[w], uniforms[step, w], nf, beta, k_cap)
            if mv is None:
                acc[step, w] = -1
                continue
            new, lp, info = mv
            lstage1 = 0.0
            if surrogate is not None:
                bs_new, bl_new = bath_weight(hyb, new, nf)
                if bs_new == 0:
                    acc[step, w] = -1
                    continue
                bs_old, bl_old = bath_weight(hyb, configs[w], nf)
                rt = float(surrogate(configs[w], *info))
                u6 = uniforms[step, w, 6]
                if not (math.log(u6) if u6 > 0 else -math.inf) < rt + bl_new - bl_old + lp:
                    acc[step, w] = -2
                    continue
                lstage1 = rt + bl_new - bl_old + lp
            nw_ = weight(model, hyb, new, trace)
            if nw_[0] == 0:
                continue
            lr = nw_[1] - cur[w][1] + lp - lstage1
            u5 = uniforms[step, w, 5]
            if (math.log(u5) if u5 > 0 else -math.inf) < lr:
                configs[w] = new
                cur[w] = nw_
                acc[step, w] = 1
        if meas_every and (step + 1) % meas_every == 0:
            n_meas += 1
            for w in range(nw):
                s = cur[w][0]
                sign_sum[w] += s
                for f in range(nf):
                    cre, ann = flavor_times(configs[w], f)
                    order_sum[w, f] += s * len(cre)
                    if not cre:
                        continue
                    M = np.linalg.inv(bath_matrix(hyb, f, cre, ann))
                    for i, tc in enumerate(cre):
                        for j, ta in enumerate(ann):
                            x, v = ta - tc, M[j, i]
                            if x < 0:
                                x, v = x + beta, -v
                            b = min(int(x / beta * n_bins), n_bins - 1)
                            g_acc[w, f, b] += s * v
            if observables:
                val, _, _ = measure(model, SeqBatch.from_lists(configs))
                sg = np.array([c[0] for c in cur], dtype=np.float64)
                obs_sum = val * sg[:, None] if obs_sum is None else obs_sum + val * sg[:, None]
    out = {"accepted": acc, "configs": configs, "sign": np.array([c[0] for c in cur]),
           "logw": np.array([c[1] for c in cur]), "trace_sign": np.array([c[2] for c in cur]),
           "trace_log": np.array([c[3] for c in cur])}
    if meas_every:
        out.update(g_acc=g_acc, sign_sum=sign_sum, order_sum=order_sum, n_meas=n_meas)
        if observables:
            out["obs_sum"] = obs_sum
    return out


def chain_da_multi(model: Model, hyb: Hyb, init, uniforms: np.ndarray, surrogate, k_cap: int = 64,
                   n_bins: int = 50, meas_every: int = 0, observables: bool = False, trace=None):
    """Multi-try delayed acceptance. uniforms [n_steps, n_walkers, tries, 7], each try's seven
    as in chain(). A null move or a stage-1 rejection is a Metropolis step that keeps the
    configuration, so per step every walker takes its tries in order from its configuration
    until one passes stage 1; that one is judged at stage 2 and ends the step, and the later
    tries are not taken. A step is thus n = 1 .. tries Metropolis steps of the walker.

    Measurement weights: the step's off-diagonal transition probability from x to y is
    c(x) K(x, y), with K the delayed-acceptance kernel and c(x) the expected number of tries
    taken from x, so the step chain is stationary in w(x) / c(x). Every meas_every steps the
    configuration each walker holds after stage 1 (before stage 2) is measured with the
    weight n of that step's tries, an unbiased estimate of c(x): sums of n * sign * O, and
    sign_sum = sum n * sign, whose ratio estimates <O> under w.

    Returns a dict: accepted [n_steps, n_walkers] (1 accepted at stage 2, 0 rejected at stage
    2 or a zero new weight, -2 no try passed stage 1), tries [n_steps, n_walkers] (n),
    counts {"proposals", "insertions", "removals", "null", "stage1_rejected"} over the tries
    taken, configs, sign / logw, and when meas_every > 0 the accumulators of chain()."""
    beta = model.p.beta
    nf = 2 * model.p.n_orb
    n_steps, nw, T, _ = uniforms.shape
    configs = [list(c) for c in init]
    cur = [weight(model, hyb, c, trace) for c in configs]
    acc = np.zeros((n_steps, nw), dtype=np.int8)
    tries = np.zeros((n_steps, nw), dtype=np.int32)
    counts = {"proposals": 0, "insertions": 0, "removals": 0, "null": 0, "stage1_rejected": 0}
    g_acc = np.zeros((nw, nf, n_bins))
    sign_sum = np.zeros(nw)
    order_sum = np.zeros((nw, nf))
    obs_sum = None
    n_meas = 0
    for step in range(n_steps):
        passed = [None] * nw
        for w in range(nw):
            n = T
            for t in range(T):
                u = uniforms[step, w, t]
                counts["proposals"] += 1
                counts["insertions" if u[0] < 0.5 else "removals"] += 1
                mv = propose(configs[w], u, nf, beta, k_cap)
                if mv is None:
                    counts["null"] += 1
                    continue
                new, lp, info = mv
                bs_new, bl_new = bath_weight(hyb, new, nf)
                if bs_new == 0:
                    counts["null"] += 1
                    continue
                bs_old, bl_old = bath_weight(hyb, configs[w], nf)
                lstage1 = float(surrogate(configs[w], *info)) + bl_new - bl_old + lp
                if not (math.log(u[6]) if u[6] > 0 else -math.inf) < lstage1:
                    counts["stage1_rejected"] += 1
                    continue
                n = t + 1
                passed[w] = (new, lp, lstage1, u[5])
                break
            tries[step, w] = n
        if meas_every and (step + 1) % meas_every == 0:
            n_meas += 1
            for w in range(nw):
                s = cur[w][0] * float(tries[step, w])
                sign_sum[w] += s
                for f in range(nf):
                    cre, ann = flavor_times(configs[w], f)
                    order_sum[w, f] += s * len(cre)
                    if not cre:
                        continue
                    M = np.linalg.inv(bath_matrix(hyb, f, cre, ann))
                    for i, tc in enumerate(cre):
                        for j, ta in enumerate(ann):
                            x, v = ta - tc, M[j, i]
                            if x < 0:
                                x, v = x + beta, -v
                            b = min(int(x / beta * n_bins), n_bins - 1)
                            g_acc[w, f, b] += s * v
            if observables:
                val, _, _ = measure(model, SeqBatch.from_lists(configs))
                sg = np.array([c[0] for c in cur], dtype=np.float64) * tries[step].astype(np.float64)
                obs_sum = val * sg[:, None] if obs_sum is None else obs_sum + val * sg[:, None]
        for w in range(nw):
            if passed[w] is None:
                acc[step, w] = -2
                continue
            new, lp, lstage1, u5 = passed[w]
            nw_ = weight(model, hyb, new, trace)
            if nw_[0] == 0:
                continue
            lr = nw_[1] - cur[w][1] + lp - lstage1
            if (math.log(u5) if u5 > 0 else -math.inf) < lr:
                configs[w] = new
                cur[w] = nw_
                acc[step, w] = 1
    out = {"accepted": acc, "tries": tries, "counts": counts, "configs": configs,
           "sign": np.array([c[0] for c in cur]), "logw": np.array([c[1] for c in cur]),
           "trace_sign": np.array([c[2] for c in cur]), "trace_log": np.array([c[3] for c in cur])}
    if meas_every:
        out.update(g_acc=g_acc, sign_sum=sign_sum, order_sum=order_sum, n_meas=n_meas)
        if observables:
            out["obs_sum"] = obs_sum
    return out


def green_function(g_acc: np.ndarray, sign_sum: np.ndarray, beta: float) -> np.ndarray:
    """G_f(tau) at the bin centres from the accumulated estimator (summed over walkers)."""
    n_bins = g_acc.shape[-1]
    tot = g_acc.sum(axis=0) if g_acc.ndim == 3 else g_acc
    return tot * (n_bins / beta ** 2) / float(np.sum(sign_sum))
