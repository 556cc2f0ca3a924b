"""Pins of the oracle's measurement at tau = beta/2 (Sec. III: local observables in the
truncated trace are measured in the middle of the imaginary-time interval).

Each test ties oracle.measure / Model.trace_obs to something outside it: the plain trace
(already pinned in test_oracle_pins.py) of a sequence with the observable written as
c^+ c operators, closed forms of the kept multiplet, and the occupation-string picture of
a density-density H_loc.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle.oracle import Model, Params, SeqBatch, classify, measure, observable_table
from tests import brute
from tests.test_oracle_pins import _random_ops, mu_half

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_degeneracies.json")))


def _layout(n):
    nf = 2 * n
    return slice(0, nf), slice(nf, nf + n), slice(nf + n + 1, nf + n + 1 + (n + 1) ** 2)


def test_observable_table_counts():
    """The table rows are n_f, n_up n_dn per orbital and sector projectors over all bitstrings."""
    for n in (1, 2, 3):
        t = observable_table(n)
        assert t.shape == (3 * n + (n + 1) ** 2, 4 ** n)
        sn, sd = slice(0, 2 * n), slice(2 * n, 3 * n)
        ss = slice(3 * n, 3 * n + (n + 1) ** 2)
        assert (t[sn].sum(axis=1) == 4 ** n / 2).all()          # each bit set in half of the states
        assert (t[sd].sum(axis=1) == 4 ** n / 4).all()
        assert (t[ss].sum(axis=0) == 1).all()                   # every state in exactly one sector


@pytest.mark.parametrize("n, kept", [(3, 4), (5, 6)])
def test_empty_sequence_kept_multiplet(n, kept):
    """No operators: the average over the kept high-spin multiplet at half filling
    (S = n/2, all orbitals singly occupied): n_f = 1/2, no double occupancy, and the
    2S + 1 states spread evenly over the sectors n_up + n_dn = n."""
    U, J = (6.0, 1.0) if n == 3 else (4.0, 1.0)
    mu = mu_half(3, U, J) if n == 3 else 4.5 * U - 10 * J
    m = Model(Params(n, U, J, mu=mu, beta=50.0))
    assert m.nkept == kept
    val, s, _ = measure(m, SeqBatch.from_lists([[]]))
    sn, sd, ss = _layout(n)
    assert s[0] == 1
    assert np.allclose(val[0, sn], 0.5, atol=1e-12)
    assert np.allclose(val[0, sd], 0.0, atol=1e-12)
    hist = val[0, ss].reshape(n + 1, n + 1)
    for u in range(n + 1):
        for d in range(n + 1):
            assert abs(hist[u, d] - (1.0 / (n + 1) if u + d == n else 0.0)) < 1e-12


def _insert_at(ops, t, new):
    """ops with the operators `new` (applied in list order) placed at time t after every op before t."""
    pos = 0
    while pos < len(ops) and ops[pos][0] < t:
        pos += 1
    return ops[:pos] + [(t, f, d) for f, d in new] + ops[pos:]


@pytest.mark.parametrize("trunc", [0.0, 1e-10])
def test_density_and_double_occupancy_as_operator_strings(trunc):
    """n_f = c_f^+ c_f and n_{a up} n_{a dn} = c^+_{a up} c_{a up} c^+_{a dn} c_{a dn}: the
    trace with these operators written into the sequence at beta/2 (the pinned plain
    trace), divided by the trace, is the measured value."""
    n, U, J, beta = 3, 4.0, 1.0, 8.0
    rng = np.random.default_rng(11)
    delta = rng.uniform(-0.2, 0.2, n)
    m = Model(Params(n, U, J, mu=mu_half(n, U, J) + 0.3, delta=tuple(delta), beta=beta, trunc_eps=trunc))
    mx = Model(Params(n, U, J, mu=mu_half(n, U, J) + 0.3, delta=tuple(delta), beta=beta, trunc_eps=trunc), "ext")
    lists = [_random_ops(rng, n, beta, 3) for _ in range(40)]
    seqs = SeqBatch.from_lists(lists)
    val, s, la = measure(m, seqs)
    sx, lax, _ = mx.trace(seqs)
    cls = classify(s, la, sx, lax)
    sn, sd, _ = _layout(n)
    checked = 0
    for i, ops in enumerate(lists):
        if cls[i] != 2:
            continue
        strings = [[(f, 0), (f, 1)] for f in range(2 * n)]
        strings += [[(2 * a, 0), (2 * a, 1), (2 * a + 1, 0), (2 * a + 1, 1)] for a in range(n)]
        alt = SeqBatch.from_lists([_insert_at(ops, 0.5 * beta, st) for st in strings])
        s2, la2, _ = m.trace(alt)
        ref = s2.astype(float) * s[i] * np.exp(la2 - la[i])
        got = np.concatenate([val[i, sn], val[i, sd]])
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-11), (i, got, ref)
        checked += 1
    assert checked >= 20


def test_identity_observable_is_the_trace():
    """O = 1 inserted anywhere leaves the trace unchanged."""
    n, U, J, beta = 3, 4.0, 1.0, 10.0
    m = Model(Params(n, U, J, mu=5.0, beta=beta, trunc_eps=1e-10))
    mx = Model(Params(n, U, J, mu=5.0, beta=beta, trunc_eps=1e-10), "ext")
    rng = np.random.default_rng(5)
    seqs = SeqBatch.from_lists([_random_ops(rng, n, beta, 4) for _ in range(60)])
    s, la, _ = m.trace(seqs)
    sx, lax, _ = mx.trace(seqs)
    cls = classify(s, la, sx, lax)
    ones = np.ones((1, 4 ** n))
    for t in (0.0, 0.31 * beta, 0.5 * beta, beta):
        so, lo = m.trace_obs(seqs, t, ones)
        reg = cls == 2
        assert reg.sum() >= 10
        assert (so[reg, 0] == s[reg]).all()
        assert np.abs(lo[reg, 0] - la[reg]).max() < 1e-10
        assert (so[cls == 0, 0] == 0).all()


def test_density_only_occupation_at_half_beta():
    """Density-density H_loc: every surviving occupation string x(tau) has a definite
    occupation at beta/2, so <n_f(beta/2)> and the sector histogram are the
    exp(-integral E_diag)-weighted averages over the strings (segment picture, Sec. II)."""
    n, U, J, mu, beta = 2, 4.0, 1.0, 3.0, 6.0
    rng = np.random.default_rng(9)
    delta = rng.uniform(-0.3, 0.3, n)
    m = Model(Params(n, U, J, mu=mu, delta=tuple(delta), beta=beta, trunc_eps=0.0, density_only=True))
    Hd = np.diag(brute.hamiltonian(n, U, J, U - 2 * J, mu, delta, density_only=True))
    E0 = Hd.min()
    table = observable_table(n)
    done = 0
    for _ in range(30):
        ops = _random_ops(rng, n, beta, 2)
        num = np.zeros(table.shape[0])
        den = 0.0
        for x0 in range(4 ** n):
            x, sgn, t_prev, expo, ok, xmid = x0, 1, 0.0, 0.0, True, None
            for (t, f, d) in ops:
                if xmid is None and t >= 0.5 * beta:
                    xmid = x
                expo += (t - t_prev) * (Hd[x] - E0)
                bit = 1 << f
                if bool(x & bit) == bool(d):
                    ok = False
                    break
                if bin(x & (bit - 1)).count("1") % 2:
                    sgn = -sgn
                x ^= bit
                t_prev = t
            if not ok or x != x0:
                continue
            if xmid is None:
                xmid = x
            expo += (beta - t_prev) * (Hd[x] - E0)
            wgt = sgn * math.exp(-expo)
            den += wgt
            num += wgt * table[:, xmid]
        val, s, _ = measure(m, SeqBatch.from_lists([ops]))
        if den == 0.0:
            assert s[0] == 0 and np.isnan(val[0]).all()
            continue
        assert np.allclose(np.delete(val[0], 3 * n), num / den, rtol=1e-10, atol=1e-12)   # all but S^2
        done += 1
    assert done >= 10


def test_histogram_and_densities_are_consistent():
    """The sector histogram sums to 1 and its mean n_up + n_dn equals sum_f <n_f>."""
    n, beta = 3, 10.0
    m = Model(Params(n, 4.0, 1.0, mu=5.0, beta=beta, trunc_eps=1e-10))
    rng = np.random.default_rng(6)
    seqs = SeqBatch.from_lists([_random_ops(rng, n, beta, 4) for _ in range(30)])
    val, s, _ = measure(m, seqs)
    sn, _, ss = _layout(n)
    ok = s != 0
    hist = val[ok][:, ss].reshape(-1, n + 1, n + 1)
    N = np.add.outer(np.arange(n + 1), np.arange(n + 1))
    assert np.allclose(hist.sum(axis=(1, 2)), 1.0, atol=1e-9)
    assert np.allclose((hist * N).sum(axis=(1, 2)), val[ok][:, sn].sum(axis=1), atol=1e-9)


def test_spin_squared_operator():
    """S^2 has the eigenvalues S(S+1), S = 0, 1/2, ..., n/2, and commutes with the
    Kanamori H_loc at U' = U - 2J (Sec. IV.A: rotationally invariant), built
    independently by Kronecker products in tests/brute.py."""
    from oracle.oracle import spin_squared
    for n in (1, 2, 3):
        S2 = spin_squared(n)
        assert np.allclose(S2, S2.T)
        ev = np.linalg.eigvalsh(S2)
        allowed = np.array([s * (s + 1) for s in np.arange(0, n / 2 + 0.25, 0.5)])
        assert np.all(np.min(np.abs(ev[:, None] - allowed[None, :]), axis=1) < 1e-10)
        H = brute.hamiltonian(n, 4.0, 1.0, 2.0, 1.3, np.linspace(0, 0.1, n))
        assert np.abs(H @ S2 - S2 @ H).max() < 1e-10
    # one orbital: |0>, |up>, |dn>, |updn> -> 0, 3/4, 3/4, 0
    assert np.allclose(np.diag(spin_squared(1)), [0, 0.75, 0.75, 0])


def _ground_sector_n(val, n):
    hist = val[3 * n + 1:].reshape(n + 1, n + 1)
    return {u + d for u in range(n + 1) for d in range(n + 1) if hist[u, d] > 1e-9}


def test_total_spin_of_atomic_ground_states_paper():
    """Sec. V (total spin): S^2 of the six-electron atomic ground states (golden file),
    measured at beta/2 on the empty sequence with the ground multiplet alone."""
    g = GOLD["five_orbital_total_spin"]
    n, U = g["n_orb"], g["U"]
    for case in g["cases"]:
        J = case["J_over_U"] * U
        delta = (case["delta_two_orbitals"],) * 2 + (0.0,) * 3
        found = False
        for mu in np.linspace(4.5 * U - 10 * J, 4.5 * U - 10 * J + 2 * U + 6 * J, 41)[1:]:
            m = Model(Params(n, U, J, mu=float(mu), delta=delta, beta=50.0, trunc_eps=1.0))
            val, s, _ = measure(m, SeqBatch.from_lists([[]]))
            if _ground_sector_n(val[0], n) == {g["electrons"]}:
                assert abs(val[0, 3 * n] - case["S2"]) < 1e-9, (case, mu, val[0, 3 * n])
                found = True
                break
        assert found, case


def test_spin_squared_as_operator_string():
    """<S^2(beta/2)> = <S_z^2 + S_z + sum_a S-_a S+_a + sum_{a != b} S-_a S+_b>: the
    exchange terms written as c^+ c^+ c c strings at beta/2 in the pinned plain trace,
    the diagonal ones measured with the diagonal observable insertion."""
    n, U, J, beta = 2, 4.0, 1.0, 6.0
    rng = np.random.default_rng(21)
    m = Model(Params(n, U, J, mu=mu_half(n, U, J) + 0.4, beta=beta, trunc_eps=0.0))
    mx = Model(Params(n, U, J, mu=mu_half(n, U, J) + 0.4, beta=beta, trunc_eps=0.0), "ext")
    lists = [_random_ops(rng, n, beta, 2) for _ in range(30)]
    seqs = SeqBatch.from_lists(lists)
    val, s, la = measure(m, seqs)
    sx, lx, _ = mx.trace(seqs)
    cls = classify(s, la, sx, lx)
    x = np.arange(4 ** n)
    nup = sum((x >> (2 * a)) & 1 for a in range(n))
    ndn = sum((x >> (2 * a + 1)) & 1 for a in range(n))
    sz = 0.5 * (nup - ndn)
    diag = sz * sz + sz + sum(((x >> (2 * a + 1)) & 1) * (1 - ((x >> (2 * a)) & 1)) for a in range(n))
    sd, ld = m.trace_obs(seqs, 0.5 * beta, diag[None, :].astype(float))
    checked = 0
    for i, ops in enumerate(lists):
        if cls[i] != 2:
            continue
        tot = sd[i, 0] * math.exp(ld[i, 0] - la[i]) * s[i]
        for a in range(n):
            for b in range(n):
                if a == b:
                    continue
                # S-_a S+_b = c^+_{a dn} c^+_{b up} c_{b dn} c_{a up}: applied right to left
                st = [(2 * a, 0), (2 * b + 1, 0), (2 * b, 1), (2 * a + 1, 1)]
                s2, l2, _ = m.trace(SeqBatch.from_lists([_insert_at(ops, 0.5 * beta, st)]))
                if s2[0] != 0:
                    tot += s2[0] * s[i] * math.exp(l2[0] - la[i])
        assert abs(val[i, 3 * n] - tot) < 1e-9 * max(1.0, abs(tot)), (i, val[i, 3 * n], tot)
        checked += 1
    assert checked >= 10
