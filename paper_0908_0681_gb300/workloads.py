"""Seeded synthetic workloads: model parameters, operator sequences and local moves.

This module only draws random numbers and arranges them into the input layout
(CSR operator sequences, per-walker move arrays). It holds none of the trace
arithmetic, so the oracle tests and the GPU path consume the very same inputs.

Workloads (the paper's parameter sets, Sec. IV.A and Sec. V):

* ``three_orbital``: 3-orbital Kanamori model, U=4, J=1, U'=U-2J, no crystal
  field, half filling mu = 5U/2 - 5J, beta=10; per flavor k ~ Uniform{0..8}
  c^+/c pairs at uniform times, sorted and alternating; the first operator of
  each flavor is a seeded coin (so many traces vanish structurally).
* ``five_orbital``: 5-orbital model, U=4, J=1, U'=U-2J, crystal field
  Uniform[-0.05, 0.05] (seed 2), mu = 4.5U - 10J, beta=50; per flavor
  k ~ Poisson(6) capped at 40; the occupation at tau=0 is drawn from the
  support of the kept high-spin multiplet (every orbital singly occupied, a
  random spin each), which fixes each flavor's first operator.
* ``seven_orbital``: 7-orbital model, U=6, J=0.7, U'=U-2J, crystal field
  Uniform[-0.1, 0.1] (seed 4), mu = 1.5(U-3J) (middle of the two-electron
  window), beta=40; per flavor k ~ Poisson(4) capped at 40; the occupation
  at tau=0 has two random orbitals singly occupied with random spins.

Moves (local updates, Sec. II): 50/50 insert/remove. Insert picks a uniform
flavor and a uniform time t1; the pair is a segment (c^+ at t1, c later) when
the flavor is empty at t1 and an anti-segment (c at t1, c^+ later) when it is
occupied (a coin when the flavor has no operators); the second time is
uniform in the gap up to the flavor's next operator, cyclically. Remove picks
a uniform flavor with at least one pair and a uniform c^+ of it; the c that
follows it cyclically goes with it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class ModelSpec:
    n_orb: int
    U: float
    J: float
    mu: float
    delta: tuple
    beta: float
    Up: float | None = None
    trunc_eps: float = 1e-10
    deg_tol: float = 1e-9
    krylov_tol: float = 1e-12

    @property
    def up(self) -> float:
        return self.U - 2.0 * self.J if self.Up is None else self.Up


@dataclass
class Workload:
    name: str
    model: ModelSpec
    start: str            # "coin" or "pattern"
    order: str            # "uniform8" or "poisson"
    lam: float = 0.0
    cap: int = 40
    pattern_singles: int = 0  # number of singly occupied orbitals at tau = 0 ("pattern")
    extra: dict = field(default_factory=dict)


def three_orbital(trunc_eps: float = 1e-10) -> Workload:
    U, J = 4.0, 1.0
    return Workload("three_orbital", ModelSpec(3, U, J, mu=2.5 * U - 5 * J, delta=(0.0,) * 3, beta=10.0,
                                               trunc_eps=trunc_eps),
                    start="coin", order="uniform8")


def five_orbital(trunc_eps: float = 1e-10) -> Workload:
    U, J = 4.0, 1.0
    delta = tuple(np.random.default_rng(2).uniform(-0.05, 0.05, 5).tolist())
    return Workload("five_orbital", ModelSpec(5, U, J, mu=4.5 * U - 10 * J, delta=delta, beta=50.0,
                                              trunc_eps=trunc_eps),
                    start="pattern", order="poisson", lam=6.0, pattern_singles=5)


def seven_orbital(trunc_eps: float = 1e-10) -> Workload:
    U, J = 6.0, 0.7
    delta = tuple(np.random.default_rng(4).uniform(-0.1, 0.1, 7).tolist())
    return Workload("seven_orbital", ModelSpec(7, U, J, mu=1.5 * (U - 3 * J), delta=delta, beta=40.0,
                                               trunc_eps=trunc_eps),
                    start="pattern", order="poisson", lam=4.0, pattern_singles=2)


WORKLOADS = {"three_orbital": three_orbital, "five_orbital": five_orbital, "seven_orbital": seven_orbital}


def five_orbital_sweep(beta: float = 50.0) -> Workload:
    """The five-orbital model at inverse temperature beta, for full CT-HYB sweeps."""
    w = five_orbital()
    m = w.model
    return Workload(f"five_orbital_sweep_beta{beta:g}", ModelSpec(m.n_orb, m.U, m.J, mu=m.mu, delta=m.delta, beta=beta),
                    start="empty", order="none")


def semicircular_hybridization(beta: float, n_flavors: int, n_tau: int = 2000, half_bandwidth: float = 2.0,
                               n_quad: int = 4096) -> np.ndarray:
    """Bath correlator of a semicircular density of states (the synthetic stand-in for a
    DMFT hybridization function), tabulated for every flavor on tau_i = i beta / n_tau:

        F(tau) = -Delta(tau) = t^2 int rho(e) e^{-tau e} / (1 + e^{-beta e}) de,
        rho(e) = 2 sqrt(D^2 - e^2) / (pi D^2),  t = D / 2,

    i.e. Delta = t^2 G of the half-filled Bethe lattice with bandwidth 2D. The integral
    is taken over e = D cos(theta) with Gauss-Legendre nodes in theta. Shape
    [n_flavors, n_tau + 1]."""
    D = float(half_bandwidth)
    t2 = (0.5 * D) ** 2
    x, wq = np.polynomial.legendre.leggauss(n_quad)
    th = 0.5 * np.pi * (x + 1.0)
    wth = 0.5 * np.pi * wq * (2.0 / np.pi) * np.sin(th) ** 2   # rho(e) de = (2/pi) sin^2(theta) dtheta
    e = D * np.cos(th)
    tau = np.linspace(0.0, beta, n_tau + 1)
    expo = -np.outer(tau, e) - np.logaddexp(0.0, -beta * e)[None, :]
    F = t2 * (np.exp(expo) * wth[None, :]).sum(axis=1)
    return np.ascontiguousarray(np.broadcast_to(F, (n_flavors, n_tau + 1)))


def sweep_uniforms(n_steps: int, n_walkers: int, seed: int) -> np.ndarray:
    """The random numbers of a run of Metropolis steps: [n_steps, n_walkers, 6] uniforms in [0, 1)."""
    return np.random.default_rng(seed).random((n_steps, n_walkers, 6))


@dataclass
class Sequences:
    """CSR operator sequences: ops of walker i are offsets[i] .. offsets[i+1]-1."""
    offsets: np.ndarray  # int32 [n+1]
    tau: np.ndarray      # float64
    flavor: np.ndarray   # uint8
    dagger: np.ndarray   # uint8 (1 = c^+, 0 = c)

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    def walker(self, i: int):
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return self.tau[a:b], self.flavor[a:b], self.dagger[a:b]

    def subset(self, idx) -> "Sequences":
        offs = [0]; t, f, d = [], [], []
        for i in idx:
            tt, ff, dd = self.walker(int(i))
            t.append(tt); f.append(ff); d.append(dd)
            offs.append(offs[-1] + len(tt))
        cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
        return Sequences(np.array(offs, dtype=np.int32), cat(t, np.float64), cat(f, np.uint8), cat(d, np.uint8))


def _flavor_times(rng, beta: float, k: int) -> np.ndarray:
    while True:
        ts = np.sort(rng.uniform(0.0, beta, 2 * k))
        if len(np.unique(ts)) == len(ts):
            return ts


def generate_sequences(w: Workload, n_walkers: int, seed: int) -> Sequences:
    """Draw n_walkers time-ordered, per-flavor alternating operator sequences."""
    rng = np.random.default_rng(seed)
    n = w.model.n_orb
    nf = 2 * n
    beta = w.model.beta
    offs = [0]
    tau_all, fl_all, dg_all = [], [], []
    for _ in range(n_walkers):
        if w.start == "pattern":
            occ0 = np.zeros(nf, dtype=np.int64)
            singles = rng.choice(n, size=w.pattern_singles, replace=False)
            for a in singles:
                occ0[2 * a + int(rng.integers(2))] = 1
        ts, fs, ds = [], [], []
        for f in range(nf):
            if w.order == "uniform8":
                k = int(rng.integers(0, 9))
            else:
                k = min(int(rng.poisson(w.lam)), w.cap)
            times = _flavor_times(rng, beta, k)
            if w.start == "coin":
                first_dag = int(rng.integers(2))
            else:
                first_dag = 0 if occ0[f] else 1  # occupied at tau=0 -> first operator is c
            for j, t in enumerate(times):
                ts.append(t); fs.append(f); ds.append(first_dag if j % 2 == 0 else 1 - first_dag)
        order = np.argsort(np.array(ts), kind="stable")
        ts = np.array(ts)[order]
        if len(np.unique(ts)) != len(ts):  # equal times across flavors: redraw is simplest
            return generate_sequences(w, n_walkers, seed + 7919)
        tau_all.append(ts); fl_all.append(np.array(fs, dtype=np.uint8)[order]); dg_all.append(np.array(ds, dtype=np.uint8)[order])
        offs.append(offs[-1] + len(ts))
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    return Sequences(np.array(offs, dtype=np.int32), cat(tau_all, np.float64), cat(fl_all, np.uint8), cat(dg_all, np.uint8))


@dataclass
class Moves:
    kind: np.ndarray     # uint8: 0 insert, 1 remove
    flavor: np.ndarray   # uint8
    t_dag: np.ndarray    # float64 (insert)
    t_ann: np.ndarray    # float64 (insert)
    rem_idx: np.ndarray  # int32 (remove: index of the c^+ inside the walker's sequence)

    def as_dict(self):
        return {"kind": self.kind, "flavor": self.flavor, "t_dag": self.t_dag, "t_ann": self.t_ann, "rem_idx": self.rem_idx}

    def subset(self, idx) -> "Moves":
        idx = np.asarray(idx, dtype=np.int64)
        return Moves(self.kind[idx], self.flavor[idx], self.t_dag[idx], self.t_ann[idx], self.rem_idx[idx])


def generate_moves(w: Workload, seqs: Sequences, seed: int) -> Moves:
    """One proposed local update per walker."""
    rng = np.random.default_rng(seed)
    nf = 2 * w.model.n_orb
    beta = w.model.beta
    n = seqs.n
    kind = np.zeros(n, np.uint8); flv = np.zeros(n, np.uint8)
    tdag = np.zeros(n, np.float64); tann = np.zeros(n, np.float64); rem = np.zeros(n, np.int32)
    for i in range(n):
        tau, fl, dg = seqs.walker(i)
        counts = np.bincount(fl, minlength=nf)
        has = np.nonzero(counts)[0]
        do_remove = len(has) > 0 and rng.random() < 0.5
        if do_remove:
            f = int(rng.choice(has))
            idx = np.nonzero((fl == f) & (dg == 1))[0]
            kind[i] = 1; flv[i] = f; rem[i] = int(rng.choice(idx))
            continue
        f = int(rng.integers(nf))
        t1 = float(rng.uniform(0.0, beta))
        mine = np.nonzero(fl == f)[0]
        if len(mine) == 0:
            occupied = bool(rng.integers(2))
            gap = beta
        else:
            ft = tau[mine]; fd = dg[mine]
            before = np.nonzero(ft < t1)[0]
            last = int(before[-1]) if len(before) else len(ft) - 1  # cyclic predecessor
            occupied = bool(fd[last] == 1)
            after = np.nonzero(ft > t1)[0]
            nxt = float(ft[after[0]]) if len(after) else float(ft[0]) + beta
            gap = nxt - t1
        while True:
            t2 = t1 + float(rng.uniform(0.0, 1.0)) * gap
            if t2 >= beta:
                t2 -= beta
            if t2 != t1 and t2 not in tau and 0.0 <= t2 < beta:
                break
        kind[i] = 0; flv[i] = f
        if occupied:   # anti-segment: c at t1, c^+ at t2
            tann[i], tdag[i] = t1, t2
        else:          # segment: c^+ at t1, c at t2
            tdag[i], tann[i] = t1, t2
    return Moves(kind, flv, tdag, tann, rem)
