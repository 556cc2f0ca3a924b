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
- Multi-try delayed acceptance (chain_da_multi): with one try it is delayed acceptance
  decision for decision; on a finite toy chain, the exact transition matrix of a step is
  stationary in pi / c (c the expected tries), so tries-weighted measurements are exact and
  unweighted ones are not; and at U = 0 the weighted G(tau) is the semicircular one.
"""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle.ctqmc import Hyb, chain, chain_da_multi, green_function, weight
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


def _guess(beta):
    def guess(ops, kind, flavor, t1, t2, seg):
        d = (t2 - t1) % beta
        return -0.3 * d if kind == 0 else 0.3 * d
    return guess


def test_multi_try_with_one_try_is_delayed_acceptance():
    """One try per step takes exactly the delayed-acceptance chain's decisions."""
    beta, nw, steps = 4.0, 6, 400
    m = Model(Params(1, 2.0, 0.0, mu=1.0, beta=beta, trunc_eps=0.0))
    hyb = Hyb(workloads.semicircular_hybridization(beta, 2, n_tau=400), beta)
    u = np.random.default_rng(21).random((steps, nw, 7))
    a = chain(m, hyb, [[] for _ in range(nw)], u, k_cap=64, surrogate=_guess(beta))
    b = chain_da_multi(m, hyb, [[] for _ in range(nw)], u[:, :, None, :], _guess(beta), k_cap=64)
    assert a["configs"] == b["configs"]
    assert ((a["accepted"] == 1) == (b["accepted"] == 1)).all()
    # chain() codes a null move -1 and a stage-1 rejection -2; with one try both are "no try passed"
    assert ((a["accepted"] < 0) == (b["accepted"] == -2)).all()
    assert (b["tries"] == 1).all()
    assert b["counts"]["stage1_rejected"] == int((a["accepted"] == -2).sum()) > 0


def _multi_try_step_matrix(pi, g, T):
    """Exact transition matrix of one multi-try delayed-acceptance step on states 0..N-1:
    uniform proposals to the other states, stage 1 min(1, e^{g(y) - g(x)}) (surrogate
    log ratio g(y) - g(x), antisymmetric), stage 2 min(1, pi(y)/pi(x) e^{-(g(y) - g(x))}),
    at most T tries, each rejected try keeping x. Returns (P, c) with c(x) the expected
    number of tries taken from x."""
    N = len(pi)
    q = (np.ones((N, N)) - np.eye(N)) / (N - 1)
    a1 = np.minimum(1.0, np.exp(g[None, :] - g[:, None]))
    a2 = np.minimum(1.0, (pi[None, :] / pi[:, None]) * np.exp(-(g[None, :] - g[:, None])))
    r = 1.0 - (q * a1).sum(1)                     # a try from x fails stage 1
    c = np.array([sum(ri ** t for t in range(T)) for ri in r])
    P = c[:, None] * q * a1 * a2
    P[np.diag_indices(N)] = 0.0
    P[np.diag_indices(N)] = 1.0 - P.sum(1)
    return P, c


def test_multi_try_weights_make_the_estimate_exact():
    """The weighting rule of chain_da_multi, checked on a finite chain by linear algebra:
    the step chain's stationary law mu is proportional to pi / c, so weighting each
    measured state by its number of tries (mean c) recovers pi exactly, while the
    unweighted step average is biased; one try (c = 1) needs no weight."""
    rng = np.random.default_rng(3)
    N = 6
    pi = rng.random(N) + 0.1
    pi /= pi.sum()
    g = np.log(pi) + rng.normal(0, 0.8, N)       # an imperfect surrogate
    for T in (1, 3, 8):
        P, c = _multi_try_step_matrix(pi, g, T)
        ev, V = np.linalg.eig(P.T)
        mu = np.real(V[:, np.argmin(np.abs(ev - 1.0))])
        mu /= mu.sum()
        weighted = mu * c / (mu * c).sum()
        assert np.abs(weighted - pi).max() < 1e-12, T
        if T == 1:
            assert np.abs(mu - pi).max() < 1e-12
        else:
            assert np.abs(mu - pi).max() > 1e-3, T


def test_multi_try_delayed_acceptance_keeps_the_distribution():
    """Four tries per step with the crude surrogate: the tries-weighted U = 0 Green's
    function is the semicircular one, and steps take more than one Metropolis step on
    average."""
    beta, nw, steps, T = 4.0, 12, 1200, 4
    m = Model(Params(1, 0.0, 0.0, mu=0.0, beta=beta, trunc_eps=0.0))
    table = workloads.semicircular_hybridization(beta, 2, n_tau=400)
    hyb = Hyb(table, beta)
    u = np.random.default_rng(13).random((steps, nw, T, 7))
    nb = 10
    out = chain_da_multi(m, hyb, [[] for _ in range(nw)], u, _guess(beta), k_cap=64, n_bins=nb, meas_every=5)
    g_w = (out["g_acc"] * (nb / beta ** 2) / out["sign_sum"][:, None, None]).mean(axis=1)
    mean, err = g_w.mean(axis=0), g_w.std(axis=0, ddof=1) / math.sqrt(nw)
    grid = np.linspace(0, beta, 401)
    exact = np.array([-np.mean(np.interp(np.linspace(b * beta / nb, (b + 1) * beta / nb, 41), grid, table[0]))
                      for b in range(nb)])
    assert np.all(np.abs(mean - exact) < 5 * err + 2e-3), (mean, exact, err)
    assert out["tries"].mean() > 1.3
    assert out["counts"]["proposals"] == int(out["tries"].sum())
