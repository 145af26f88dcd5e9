"""Chain post-processing on the host (Sec. 2 / 2.1: discard a burn-in
fraction, pool the chains, summarise the posterior).

Effective sample size: the multi-chain estimator of Gelman et al. (BDA3,
Sec. 11.5) in the form of Vehtari et al. (2021): autocorrelations from the
chains' FFT autocovariances combined with the within/between-chain variance,
summed in pairs while the pair sums stay positive and are made monotone
(Geyer's initial monotone sequence).  MCSE of the mean = sd / sqrt(ESS).
Split-R-hat: chains split in halves, sqrt(var+ / W).
"""
from __future__ import annotations

import numpy as np


def _autocov(x):
    """Autocovariance of each column of x [n][m] at lags 0..n-1 (biased)."""
    n = x.shape[0]
    xc = x - x.mean(axis=0, keepdims=True)
    size = 1 << int(np.ceil(np.log2(2 * n)))
    f = np.fft.rfft(xc, n=size, axis=0)
    ac = np.fft.irfft(f * np.conj(f), n=size, axis=0)[:n]
    return ac / n


def ess(samples):
    """Multi-chain effective sample size of samples [steps][chains]."""
    x = np.asarray(samples, dtype=np.float64)
    n, m = x.shape
    if n < 4:
        return float(n * m)
    acov = _autocov(x)
    chain_var = acov[0] * n / (n - 1.0)
    W = chain_var.mean()
    B = n * x.mean(axis=0).var(ddof=1) if m > 1 else 0.0
    var_plus = (n - 1.0) / n * W + B / n
    if var_plus <= 0:
        return float(n * m)
    rho = 1.0 - (W - acov.mean(axis=1)) / var_plus
    rho[0] = 1.0
    tau = -1.0
    prev = np.inf
    t = 0
    while t + 1 < n:
        pair = rho[t] + rho[t + 1]
        if pair <= 0:
            break
        pair = min(pair, prev)  # monotone
        tau += 2.0 * pair
        prev = pair
        t += 2
    return float(n * m / max(tau, 1e-12))


def split_rhat(samples):
    x = np.asarray(samples, dtype=np.float64)
    n = x.shape[0] // 2
    if n < 2:
        return float("nan")
    halves = np.concatenate([x[:n], x[n:2 * n]], axis=1)
    W = halves.var(axis=0, ddof=1).mean()
    B = n * halves.mean(axis=0).var(ddof=1)
    var_plus = (n - 1.0) / n * W + B / n
    return float(np.sqrt(var_plus / W)) if W > 0 else float("nan")


def mcse_quantile(samples, prob):
    """Monte Carlo standard error of the prob-quantile of samples
    [steps][chains], after Vehtari et al. (2021): the effective size S of the
    indicator x <= q gives the spread sqrt(prob (1 - prob) / S) of the
    quantile's level, and half the width of the pooled-sample interval
    between the levels prob -+ that spread is the standard error (their Beta
    interval in its normal limit)."""
    x = np.asarray(samples, dtype=np.float64)
    q = np.quantile(x, prob)
    s_eff = ess((x <= q).astype(np.float64))
    d = np.sqrt(prob * (1.0 - prob) / max(s_eff, 1.0))
    lo, hi = max(prob - d, 0.0), min(prob + d, 1.0)
    return float(0.5 * (np.quantile(x, hi) - np.quantile(x, lo)))


def summarize(samples, burn_frac=0.25, names=None):
    """samples [steps][P][chains] -> per-parameter mean, sd, equal-tailed 95%
    interval, ESS, MCSE of the mean and split-R-hat after burn-in."""
    s = np.asarray(samples, dtype=np.float64)
    kept = s[int(np.floor(burn_frac * s.shape[0])):]
    out = []
    for j in range(s.shape[1]):
        x = kept[:, j, :]
        e = ess(x)
        sd = float(x.std(ddof=1))
        out.append({
            "name": names[j] if names else f"p{j}",
            "mean": float(x.mean()), "sd": sd,
            "q025": float(np.quantile(x, 0.025)), "q975": float(np.quantile(x, 0.975)),
            "ess": e, "mcse": sd / np.sqrt(e), "rhat": split_rhat(x),
            "mcse_q025": mcse_quantile(x, 0.025), "mcse_q975": mcse_quantile(x, 0.975),
        })
    return out
