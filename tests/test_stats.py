"""The host-side chain summaries (ESS, split-R-hat) against the AR(1) closed
form and the oracle's single-chain estimator."""
import numpy as np
import pytest

from oracle import mcmc
from paper_1605_04718_gb300 import stats


def _ar1(phi, n, m, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((n, m))
    x = np.empty((n, m))
    x[0] = e[0] / np.sqrt(1 - phi**2)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    return x


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.9])
def test_ess_of_ar1_chains(phi):
    n, m = 4000, 16
    x = _ar1(phi, n, m, int(phi * 100))
    expect = n * m * (1 - phi) / (1 + phi)
    assert stats.ess(x) == pytest.approx(expect, rel=0.15)
    oracle_total = sum(mcmc.ess_plain(x[:, k]) for k in range(m))
    assert stats.ess(x) == pytest.approx(oracle_total, rel=0.1)


def test_rhat_detects_unmixed_chains():
    x = _ar1(0.5, 2000, 8, 1)
    assert stats.split_rhat(x) < 1.01
    y = x + np.arange(8)[None, :]  # chains stuck at different levels
    assert stats.split_rhat(y) > 1.5


def test_summarize_matches_pooled_quantiles():
    rng = np.random.default_rng(0)
    s = rng.standard_normal((1000, 2, 8)) * np.array([1.0, 3.0])[None, :, None]
    out = stats.summarize(s, burn_frac=0.2, names=["a", "b"])
    assert out[1]["name"] == "b"
    assert out[0]["q025"] == pytest.approx(-1.96, abs=0.1)
    assert out[1]["sd"] == pytest.approx(3.0, rel=0.05)
    assert out[0]["ess"] == pytest.approx(800 * 8, rel=0.15)


@pytest.mark.parametrize("prob", [0.025, 0.5, 0.975])
def test_quantile_mcse_of_independent_normals(prob):
    """For n independent N(0, 1) draws the quantile's standard error is
    sqrt(p (1 - p) / n) / phi(z_p) (the asymptotic variance of a sample
    quantile); the estimator must reproduce it, and the spread of the
    quantile over repeated samples must match it."""
    from statistics import NormalDist
    n, m = 4000, 8
    nd = NormalDist()
    z = nd.inv_cdf(prob)
    expect = np.sqrt(prob * (1 - prob) / (n * m)) / nd.pdf(z)
    rng = np.random.default_rng(int(1000 * prob))
    got = [stats.mcse_quantile(rng.standard_normal((n, m)), prob) for _ in range(3)]
    assert np.mean(got) == pytest.approx(expect, rel=0.15)
    reps = [np.quantile(rng.standard_normal((n, m)), prob) for _ in range(200)]
    assert np.std(reps) == pytest.approx(expect, rel=0.2)


def test_quantile_mcse_grows_with_autocorrelation():
    """AR(1) chains with coefficient 0.9 carry (1 - 0.9)/(1 + 0.9) of the
    information of independent draws: the quantile's standard error grows
    by about sqrt(19)."""
    x = _ar1(0.9, 8000, 8, 3) * np.sqrt(1 - 0.81)  # unit marginal variance
    y = np.random.default_rng(4).standard_normal((8000, 8))
    r = stats.mcse_quantile(x, 0.5) / stats.mcse_quantile(y, 0.5)
    assert r == pytest.approx(np.sqrt(19.0), rel=0.3)
