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


def test_single_chain_and_short_series():
    rng = np.random.default_rng(3)
    r = binning_analysis(rng.normal(size=20))
    assert set(r["errors"]) == {1, 2, 4, 5, 10}
    assert r["error"] == r["errors"][2]
