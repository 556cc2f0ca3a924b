"""Binning analysis of correlated Monte Carlo series (host logic of the sweep's error bars)."""
import math

import numpy as np

from paper_0908_0681_gb300.engine import binning_analysis


def _ar1(rng, n_chains, n_t, rho):
    x = np.empty((n_chains, n_t))
    x[:, 0] = rng.normal(size=n_chains)
    eps = rng.normal(size=(n_chains, n_t)) * math.sqrt(1 - rho * rho)
    for t in range(1, n_t):
        x[:, t] = rho * x[:, t - 1] + eps[:, t]
    return x


def test_uncorrelated_series_gives_the_naive_error():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(64, 512))
    r = binning_analysis(x)
    naive = 1 / math.sqrt(x.size)
    for b, e in r["errors"].items():
        if x.shape[1] // b >= 8:
            assert abs(e / naive - 1) < 0.2, (b, e, naive)
    assert abs(r["tau_int"] - 0.5) < 0.15


def test_ar1_error_reaches_the_exact_variance_of_the_mean():
    """AR(1) with coefficient rho and unit variance: var(mean) -> (1 + rho) / (1 - rho) / N,
    tau_int = (1 + rho) / (2 (1 - rho)). Binning must climb from the naive error to it."""
    rho = 0.8
    rng = np.random.default_rng(2)
    x = _ar1(rng, 256, 1024, rho)
    r = binning_analysis(x)
    exact = math.sqrt((1 + rho) / (1 - rho) / x.size)
    assert r["errors"][1] < 0.5 * exact
    assert abs(r["error"] / exact - 1) < 0.15, (r["error"], exact)
    assert abs(r["tau_int"] / ((1 + rho) / (2 * (1 - rho))) - 1) < 0.3
    assert r["plateau"]


def test_chains_shorter_than_the_autocorrelation_time():
    """Many independent chains, each shorter than its autocorrelation time: the whole-chain
    bins still give the right error, and the missing plateau is reported."""
    rho = 0.995
    rng = np.random.default_rng(4)
    x = _ar1(rng, 2000, 64, rho)
    r = binning_analysis(x)
    assert not r["plateau"]
    # exact variance of a 64-step AR(1) mean started in equilibrium
    n = x.shape[1]
    k = np.arange(1, n)
    var1 = (1 + 2 * np.sum((1 - k / n) * rho ** k)) / n
    exact = math.sqrt(var1 / x.shape[0])
    assert abs(r["error"] / exact - 1) < 0.1, (r["error"], exact)


def test_single_chain_and_short_series():
    rng = np.random.default_rng(3)
    r = binning_analysis(rng.normal(size=20))
    assert set(r["errors"]) == {1, 2, 4, 5, 10}
    assert r["error"] == r["errors"][2]
