"""Segment-picture local trace of the density-density H_loc (test infrastructure only).

Only the tests import this module; the product library never calls it.

Without spin flip and pair hopping, H_loc of Eq. (H_loc) is diagonal in the
occupation basis, and Sec. II's segment formulation applies: every flavor's
operators, taken in time order, alternate between c^+ and c, so the occupation of
each flavor along [0, beta) is a set of segments, and the local trace is a sum over
the initial occupations x(0) (fixed by the first operator of every flavor that has
operators, free for the others) of

    (JW sign) * exp( -sum_f eps_f L_f - sum_{f<g} U_fg O_fg ),

  L_f     total occupied time of flavor f,
  O_fg    time during which f and g are both occupied,
  eps_f   -(mu + Delta_a) for f = 2a + s,
  U_fg    U for the two spins of one orbital, U' for opposite spins of two orbitals,
          U' - J for equal spins of two orbitals,

the exponent being -integral of E_diag(x(tau)). The Jordan-Wigner sign of an
operator on flavor f is (-1) to the number of occupied flavors below f just before
it. The truncated trace keeps the initial occupations of the kept multiplets: the
occupation states x with exp(-beta (E_x - E0)) >= trunc_eps, E0 the lowest E_x,
whole multiplets (energies within deg_tol max(1, |E|) count as one level).

This evaluation is independent of the oracle's matrix exponentials: it only
measures segment lengths and overlaps.
"""
from __future__ import annotations

import math

import numpy as np


def _pair_energy(n_orb: int, U: float, J: float, Up: float):
    nf = 2 * n_orb
    W = np.zeros((nf, nf))
    for f in range(nf):
        for g in range(f + 1, nf):
            a, s, b, t = f // 2, f % 2, g // 2, g % 2
            if a == b:
                W[f, g] = U
            elif s != t:
                W[f, g] = Up
            else:
                W[f, g] = Up - J
    return W


class SegmentTrace:
    """Local trace of the density-density model from segment lengths and overlaps."""

    def __init__(self, n_orb: int, U: float, J: float, mu: float, delta, beta: float, Up: float | None = None,
                 trunc_eps: float = 1e-10, deg_tol: float = 1e-9):
        self.n_orb, self.nf, self.beta = n_orb, 2 * n_orb, beta
        Up = U - 2.0 * J if Up is None else Up
        d = np.zeros(n_orb)
        if len(delta):
            d[:] = np.asarray(delta, dtype=np.float64)
        self.eps = np.array([-(mu + d[f // 2]) for f in range(self.nf)])
        self.W = _pair_energy(n_orb, U, J, Up)
        occ = ((np.arange(1 << self.nf)[:, None] >> np.arange(self.nf)) & 1).astype(np.float64)
        self.E = occ @ self.eps + np.einsum("xf,fg,xg->x", occ, self.W, occ)
        self.E0 = float(self.E.min())
        # kept multiplets: sorted levels, grouped within deg_tol, kept by their lowest energy
        order = np.argsort(self.E, kind="stable")
        kept = np.zeros(1 << self.nf, dtype=bool)
        i = 0
        while i < len(order):
            e = self.E[order[i]]
            j = i
            while j < len(order) and self.E[order[j]] - e <= deg_tol * max(1.0, abs(e)):
                j += 1
            if math.exp(-beta * (e - self.E0)) >= trunc_eps:
                kept[order[i:j]] = True
            i = j
        self.kept = kept
        self.n_kept = int(kept.sum())

    def __call__(self, ops):
        """(sign in {-1, 0, 1}, log|T|) of a time-ordered list of (tau, flavor, dagger)."""
        nf, beta = self.nf, self.beta
        per = [[(t, d) for (t, f, d) in ops if f == g] for g in range(nf)]
        fixed = {}
        for g in range(nf):
            if not per[g]:
                continue
            ds = [d for _, d in per[g]]
            if any(ds[k] == ds[k + 1] for k in range(len(ds) - 1)) or ds[0] == ds[-1]:
                return 0, -math.inf        # Pauli: no alternating occupation string
            fixed[g] = 0 if ds[0] == 1 else 1
        free = [g for g in range(nf) if g not in fixed]
        total = 0.0
        for bits in range(1 << len(free)):
            x0 = sum(v << g for g, v in fixed.items()) + sum(((bits >> i) & 1) << g for i, g in enumerate(free))
            if not self.kept[x0]:
                continue
            segs = [self._segments(per[g], (x0 >> g) & 1) for g in range(nf)]
            L = np.array([sum(b - a for a, b in s) for s in segs])
            expo = float(self.eps @ L)
            for f in range(nf):
                for g in range(f + 1, nf):
                    if self.W[f, g] != 0.0 and L[f] > 0 and L[g] > 0:
                        expo += self.W[f, g] * _overlap(segs[f], segs[g])
            sign = 1
            for (t, f, d) in ops:
                below = sum(_occupied_before(segs[g], t) for g in range(f))
                if below % 2:
                    sign = -sign
            total += sign * math.exp(-(expo - beta * self.E0))
        if total == 0.0:
            return 0, -math.inf
        return (1 if total > 0 else -1), math.log(abs(total)) - beta * self.E0

    def _segments(self, ops_g, occ0):
        """Occupied intervals [a, b) of one flavor on [0, beta)."""
        beta = self.beta
        if not ops_g:
            return [(0.0, beta)] if occ0 else []
        out, start = [], 0.0 if occ0 else None
        for t, d in ops_g:
            if d == 1:
                start = t
            else:
                out.append((start, t))
                start = None
        if start is not None:
            out.append((start, beta))
        return out


def _overlap(sa, sb) -> float:
    tot = 0.0
    for a0, a1 in sa:
        for b0, b1 in sb:
            lo, hi = max(a0, b0), min(a1, b1)
            if hi > lo:
                tot += hi - lo
    return tot


def _occupied_before(segs, t) -> int:
    """Occupation just before time t (the operators of other flavors sit at other times)."""
    return int(any(a < t <= b for a, b in segs))
