"""Pins of the CT-HYB chain oracle (oracle/ctqmc.py) against facts outside it.

- The first-order term of Z/Z_bath for an impurity coupled to one bath level equals
  the V^2 coefficient of the exact partition function (full-space diagonalisation
  of impurity + bath): fixes the argument, the sign and the normalisation of the
  bath factor and the time order of the trace (Eq. (weight_strong) at k = 1).
- Without interaction the flavors are independent: weights factorise over flavors
  configuration by configuration, and a single flavor's weights are positive. This
  fixes the permutation sign across flavors and inside one flavor at k >= 2.
- Without interaction and with the semicircular bath, the impurity Green's function is
  the semicircular one, G(tau) = Delta(tau) / t^2 = -F(tau) / t^2 (Bethe lattice at
  U = 0): fixes the proposal probabilities, the acceptance rule and the G estimator
  of the whole chain (statistical, 5 standard errors over independent walkers).
- The tabulated semicircular bath itself against an independent adaptive quadrature.
"""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle.ctqmc import Hyb, chain, green_function, weight
from oracle.oracle import Model, Params
from paper_0908_0681_gb300 import workloads
from tests import brute


def test_semicircular_table_against_quadrature():
    beta = 7.0
    F = workloads.semicircular_hybridization(beta, 1, n_tau=700)[0]
    D = 2.0
    for i in (0, 50, 350, 612, 700):
        tau = beta * i / 700

        def f(e):
            return 2 * math.sqrt(D * D - e * e) / (math.pi * D * D) * math.exp(-tau * e) / (1 + math.exp(-beta * e))

        ref = (0.5 * D) ** 2 * scipy.integrate.quad(f, -D, D, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
        assert abs(F[i] - ref) < 1e-12
    assert abs(F[0] + F[-1] - 1.0) < 1e-12            # G(0+) + G(beta-) = -1 with t = 1
    assert np.abs(F - F[::-1]).max() < 1e-12          # particle-hole symmetric bath


def _gl_triangle(n, beta, fn):
    """int_0^beta ds int_s^beta dt fn(s, t) by Gauss-Legendre on the mapped square."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    tot = 0.0
    for a, wa in zip(x, w):
        s = beta * a
        for b, wb in zip(x, w):
            t = s + (beta - s) * b
            tot += wa * wb * beta * (beta - s) * fn(s, t)
    return tot


def test_first_order_weight_matches_exact_diagonalisation():
    """Z/Z_bath = Z_loc + V^2 Z_2 + O(V^4); Z_2 = int int w(c^+ at t', c at t) dt dt' / V^2."""
    U, mu, beta, eps = 2.3, 0.4, 3.0, 0.7
    m = Model(Params(1, U, 0.0, mu=mu, beta=beta, trunc_eps=0.0))
    n_tau = 20000
    tau = np.linspace(0.0, beta, n_tau + 1)
    table = np.zeros((2, n_tau + 1))
    table[0] = np.exp(-tau * eps) / (1.0 + math.exp(-beta * eps))   # flavor 0 couples to the level; V^2 = 1
    hyb = Hyb(table, beta)

    def w1(tc, ta):
        ops = sorted([(tc, 0, 1), (ta, 0, 0)])
        s, lw, _, _ = weight(m, hyb, ops)
        return s * math.exp(lw)

    # t' = creator time later than the annihilator time, and the other way round
    z2 = _gl_triangle(48, beta, lambda s, t: w1(t, s)) + _gl_triangle(48, beta, lambda s, t: w1(s, t))
    # exact: impurity flavors 0, 1 and the bath level as flavor 2 (flavor 3 idle)
    c = brute.fermion_ops(2)
    cd = [x.T for x in c]
    n = [cd[f] @ c[f] for f in range(4)]
    H0 = U * n[0] @ n[1] - mu * (n[0] + n[1]) + eps * n[2]
    hop = cd[0] @ c[2] + cd[2] @ c[0]
    zb = 2.0 * (1.0 + math.exp(-beta * eps))

    def coef(V):
        E = np.linalg.eigvalsh(H0 + V * hop)
        E0 = np.linalg.eigvalsh(H0)
        return (np.exp(-beta * E).sum() - np.exp(-beta * E0).sum()) / (zb * V * V)

    V = 0.02
    exact = (4.0 * coef(V / 2) - coef(V)) / 3.0
    assert abs(z2 / exact - 1.0) < 2e-6, (z2, exact)


def _random_config(rng, flavors, beta, kmax, first=None):
    ops = []
    for f in flavors:
        k = int(rng.integers(1, kmax + 1))
        ts = np.sort(rng.uniform(0, beta, 2 * k))
        d0 = int(rng.integers(2)) if first is None else first
        ops += [(float(t), f, d0 if j % 2 == 0 else 1 - d0) for j, t in enumerate(ts)]
    return sorted(ops)


def test_weights_factorise_over_flavors_without_interaction():
    """U = 0: w(c_up + c_dn) w(empty) = w(c_up) w(c_dn), signs included."""
    beta = 4.0
    m = Model(Params(1, 0.0, 0.0, mu=0.3, beta=beta, trunc_eps=0.0))
    rng = np.random.default_rng(3)
    tau = np.linspace(0, beta, 4001)
    table = np.array([0.6 * np.exp(-0.4 * tau) / (1 + math.exp(-0.4 * beta)) + 0.3 * np.exp(0.9 * tau) / (1 + math.exp(0.9 * beta)),
                      0.5 * np.exp(-1.1 * tau) / (1 + math.exp(-1.1 * beta))])
    hyb = Hyb(table, beta)
    s0, l0, _, _ = weight(m, hyb, [])
    checked = 0
    for _ in range(60):
        up = _random_config(rng, [0], beta, 3)
        dn = _random_config(rng, [1], beta, 3)
        sa, la, _, _ = weight(m, hyb, up)
        sb, lb, _, _ = weight(m, hyb, dn)
        sc, lc, _, _ = weight(m, hyb, sorted(up + dn))
        assert sc * s0 == sa * sb
        if sc != 0:
            assert abs((lc + l0) - (la + lb)) < 1e-10
            checked += 1
    assert checked > 40


def test_single_flavor_weights_positive_without_interaction():
    beta = 5.0
    m = Model(Params(1, 0.0, 0.0, mu=-0.2, beta=beta, trunc_eps=0.0))
    tau = np.linspace(0, beta, 4001)
    table = np.array([0.7 * np.exp(-0.5 * tau) / (1 + math.exp(-0.5 * beta)) + 0.2 * np.exp(1.3 * tau) / (1 + math.exp(1.3 * beta)),
                      np.zeros_like(tau)])
    hyb = Hyb(table, beta)
    rng = np.random.default_rng(4)
    for _ in range(80):
        ops = _random_config(rng, [0], beta, 5)
        s, lw, _, _ = weight(m, hyb, ops)
        assert s == 1, ops


@pytest.mark.slow
def test_chain_reproduces_semicircular_green_function():
    """One orbital, U = 0, mu = 0, semicircular bath: G(tau) = -F(tau) (t = 1)."""
    beta, nw, steps = 4.0, 12, 2500
    m = Model(Params(1, 0.0, 0.0, mu=0.0, beta=beta, trunc_eps=0.0))
    table = workloads.semicircular_hybridization(beta, 2, n_tau=400)
    hyb = Hyb(table, beta)
    u = workloads.sweep_uniforms(steps, nw, seed=11)
    nb = 10
    out = chain(m, hyb, [[] for _ in range(nw)], u, k_cap=64, n_bins=nb, meas_every=5)
    assert (out["sign"] == 1).all()
    # per-walker estimates (independent chains) -> mean and standard error per bin
    g_w = out["g_acc"] * (nb / beta ** 2) / out["sign_sum"][:, None, None]     # [nw, nf, nb]
    g_w = g_w.mean(axis=1)                                                    # both spins
    mean, err = g_w.mean(axis=0), g_w.std(axis=0, ddof=1) / math.sqrt(nw)
    centres = (np.arange(nb) + 0.5) * beta / nb
    # exact bin average of -F over each bin
    grid = np.linspace(0, beta, 401)
    exact = np.array([-np.mean(np.interp(np.linspace(b * beta / nb, (b + 1) * beta / nb, 41), grid, table[0]))
                      for b in range(nb)])
    assert np.all(np.abs(mean - exact) < 5 * err + 2e-3), (mean, exact, err, centres)
    # G(tau) is negative and symmetric about beta/2 at half filling
    assert (mean < 0).all()
    pooled = green_function(out["g_acc"], out["sign_sum"], beta)
    assert pooled.shape == (2, nb)


@pytest.mark.slow
def test_delayed_acceptance_keeps_the_distribution():
    """Delayed acceptance with a crude surrogate (a linear guess in the pair's length)
    samples the same distribution: the U = 0 Green's function is still semicircular,
    and stage 1 rejects a share of the proposals before any trace is evaluated."""
    beta, nw, steps = 4.0, 12, 2500
    m = Model(Params(1, 0.0, 0.0, mu=0.0, beta=beta, trunc_eps=0.0))
    table = workloads.semicircular_hybridization(beta, 2, n_tau=400)
    hyb = Hyb(table, beta)
    u = np.random.default_rng(12).random((steps, nw, 7))
    nb = 10

    def guess(ops, kind, flavor, t1, t2, seg):
        d = (t2 - t1) % beta
        return -0.3 * d if kind == 0 else 0.3 * d

    out = chain(m, hyb, [[] for _ in range(nw)], u, k_cap=64, n_bins=nb, meas_every=5, surrogate=guess)
    g_w = (out["g_acc"] * (nb / beta ** 2) / out["sign_sum"][:, None, None]).mean(axis=1)
    mean, err = g_w.mean(axis=0), g_w.std(axis=0, ddof=1) / math.sqrt(nw)
    grid = np.linspace(0, beta, 401)
    exact = np.array([-np.mean(np.interp(np.linspace(b * beta / nb, (b + 1) * beta / nb, 41), grid, table[0]))
                      for b in range(nb)])
    assert np.all(np.abs(mean - exact) < 5 * err + 2e-3), (mean, exact, err)
    assert (out["accepted"] == -2).mean() > 0.05
