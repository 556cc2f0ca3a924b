"""The segment-picture trace of the density-density model (oracle/segment.py) against the
oracle's matrix-exponential trace, and the oracle chain run on either.

The segment picture (Sec. II) measures segment lengths and overlaps; the oracle
multiplies blockwise matrix exponentials. For density-density H_loc both are the same
trace, truncated or not, so they pin each other: a wrong interaction coefficient,
chemical-potential sign, Jordan-Wigner count or kept set shows up as a mismatch.
"""
import math

import numpy as np
import pytest

from oracle.ctqmc import Hyb, chain
from oracle.oracle import Model, Params, SeqBatch
from oracle.segment import SegmentTrace
from paper_0908_0681_gb300 import workloads


def _random_ops(rng, n, beta, kmax, unbalanced=False):
    ops = []
    for f in range(2 * n):
        k = int(rng.integers(0, kmax + 1))
        ts = np.sort(rng.uniform(0, beta, 2 * k + (1 if unbalanced and f == 0 else 0)))
        first = int(rng.integers(2))
        for j, t in enumerate(ts):
            ops.append((float(t), f, first if j % 2 == 0 else 1 - first))
    ops.sort()
    return ops


@pytest.mark.parametrize("n,trunc_eps,beta", [(1, 0.0, 5.0), (2, 0.0, 4.0), (3, 0.0, 6.0), (3, 1e-10, 10.0),
                                              (3, 1e-3, 10.0), (4, 1e-6, 8.0)])
def test_segment_trace_equals_matrix_trace(n, trunc_eps, beta):
    rng = np.random.default_rng(7 + n)
    U, J = 4.0, 0.8
    mu = 0.5 * (U + (n - 1) * (2 * U - 5 * J))
    delta = tuple(rng.uniform(-0.3, 0.3, n))
    P = Params(n, U, J, mu=mu, delta=delta, beta=beta, trunc_eps=trunc_eps, density_only=True)
    m = Model(P)
    seg = SegmentTrace(n, U, J, mu, delta, beta, trunc_eps=trunc_eps)
    assert seg.n_kept == m.nkept
    nonzero = 0
    for trial in range(30 if trunc_eps == 0.0 else 300):
        ops = _random_ops(rng, n, beta, 3 if trunc_eps == 0.0 else 1, unbalanced=(trial % 10 == 9))
        s, la, _ = m.trace(SeqBatch.from_lists([ops]))
        s2, l2 = seg(ops)
        assert int(s[0]) == s2, (trial, ops)
        if s2 != 0:
            nonzero += 1
            assert abs(float(la[0]) - l2) < 1e-10, (trial, float(la[0]), l2)
    assert nonzero >= 5


def test_segment_trace_closed_forms():
    """One orbital: Z for the empty sequence; a single up segment of length l weighs
    e^{-l eps} times the empty-down-flavor and full-down-flavor alternatives."""
    U, mu, beta = 3.0, 1.2, 5.0
    seg = SegmentTrace(1, U, 0.0, mu, (0.0,), beta, trunc_eps=0.0)
    Z = 1 + 2 * math.exp(beta * mu) + math.exp(-beta * (U - 2 * mu))
    s, l = seg([])
    assert s == 1 and abs(l - math.log(Z)) < 1e-12
    t1, t2 = 1.0, 3.5
    s, l = seg([(t1, 0, 1), (t2, 0, 0)])
    L = t2 - t1
    ref = math.exp(mu * L) * (1 + math.exp(mu * beta - U * L))
    assert s == 1 and abs(l - math.log(ref)) < 1e-12
    # Jordan-Wigner: only the operators of flavor 1 see flavor 0 below them. The c_1^+ at
    # 1.0 finds flavor 0 occupied (-1), the c_1 at 3.0 finds it empty (+1).
    s, _ = seg([(0.5, 0, 1), (1.0, 1, 1), (2.0, 0, 0), (3.0, 1, 0)])
    assert s == -1


def test_chain_on_segment_trace_matches_matrix_trace():
    """The oracle chain with the segment-picture trace takes the same decisions as with
    the matrix trace (three orbitals, density-density, beta = 10, ground multiplet)."""
    w = workloads.three_orbital()
    sp = w.model
    P = Params(sp.n_orb, sp.U, sp.J, Up=sp.up, mu=sp.mu, delta=sp.delta, beta=sp.beta, trunc_eps=sp.trunc_eps,
               deg_tol=sp.deg_tol, density_only=True)
    m = Model(P)
    seg = SegmentTrace(sp.n_orb, sp.U, sp.J, sp.mu, sp.delta, sp.beta, Up=sp.up, trunc_eps=sp.trunc_eps,
                       deg_tol=sp.deg_tol)
    hyb = Hyb(workloads.semicircular_hybridization(sp.beta, 6, n_tau=2000), sp.beta)
    u = workloads.sweep_uniforms(150, 4, seed=31)
    a = chain(m, hyb, [[] for _ in range(4)], u, k_cap=16, n_bins=10, meas_every=5)
    b = chain(m, hyb, [[] for _ in range(4)], u, k_cap=16, n_bins=10, meas_every=5, trace=seg)
    assert (a["accepted"] == b["accepted"]).all()
    assert a["configs"] == b["configs"]
    assert (a["accepted"] == 1).sum() > 20
    assert np.abs(a["trace_log"] - b["trace_log"]).max() < 1e-9
    assert np.allclose(a["g_acc"], b["g_acc"])
