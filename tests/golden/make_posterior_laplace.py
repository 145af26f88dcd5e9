"""Gauss-Newton (Laplace) approximation of the posterior of the 128^2
fixed-domain workload, computed with the FP64 oracle only, written to
``posterior_laplace_rd2d_n128.txt`` beside this script.

The posterior (Sec. 2, eq. (bayes)) over eta = log(a, b, d, gamma) is
proportional to exp(-Phi(eta)) N(eta; log theta_0, 0.5^2 I) with
Phi = |y - G(eta)|^2 / (2 sigma^2) (eq. (logl)).  Near its mode it is close
to a Gaussian with precision H = J^T J / sigma^2 + I / 0.5^2, J = dG/deta
the Jacobian of the observed fields (central differences of oracle solves,
step 2e-4 in eta), and mode eta_true - H^-1 grad, grad = -J^T (y - G) /
sigma^2 + (eta - log theta_0) / 0.5^2 at eta_true (one Gauss-Newton step
from the true parameters).  The tests draw parameter vectors from this
Gaussian to spot-check Phi over the region the posterior occupies.

Usage:  python tests/golden/make_posterior_laplace.py   (about a minute on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import rd_synth  # noqa: E402

NAME = "rd2d_n128"
OUT = os.path.join(HERE, f"posterior_laplace_{NAME}.txt")
STEP = 2e-4
SIGMA_LOG = 0.5


def main():
    spec = rd_synth.DATASETS[NAME]
    ds = np.load(os.path.join(ROOT, "data", f"{NAME}.npz"))
    n = spec["n"]
    P = oracle.Problem(2, n, spec["tau"], spec["n_steps"], ds["u0"].astype(np.float64),
                       ds["v0"].astype(np.float64), y=ds["y"].astype(np.float64),
                       obs_steps=ds["obs_steps"], field_mask=spec["field_mask"],
                       sigma=spec["sigma"])
    eta0 = np.log(np.asarray(spec["theta"][:4]))
    rows = [eta0]
    for j in range(4):
        for s in (+1, -1):
            e = eta0.copy()
            e[j] += s * STEP
            rows.append(e)
    rows = np.array(rows)
    th = np.concatenate([np.exp(rows), np.zeros((len(rows), 1))], 1)
    t0 = time.time()
    _, st, fields = P.forward_batch(th, want_fields=True)
    assert np.all(st == 0)
    G = fields.reshape(len(rows), -1)  # both fields observed at the final step
    y = ds["y"].astype(np.float64).reshape(-1)
    sigma = spec["sigma"]
    J = np.stack([(G[1 + 2 * j] - G[2 + 2 * j]) / (2 * STEP) for j in range(4)], 1)
    H = J.T @ J / sigma**2 + np.eye(4) / SIGMA_LOG**2
    grad = -J.T @ (y - G[0]) / sigma**2  # prior gradient is zero at eta0 = log medians
    mode = eta0 - np.linalg.solve(H, grad)
    cov = np.linalg.inv(H)
    with open(OUT, "w") as f:
        f.write("# Gauss-Newton Laplace approximation of the posterior over log(a, b, d, gamma)\n")
        f.write(f"# workload {NAME}: {n}^2, tau {spec['tau']}, {spec['n_steps']} steps, "
                f"sigma {sigma}, log-normal priors (median = true values, sigma_log 0.5)\n")
        f.write("# written by tests/golden/make_posterior_laplace.py from FP64 oracle solves "
                f"({time.time() - t0:.0f} s)\n")
        f.write("# line 1: mode (log units); lines 2-5: covariance (log units)\n")
        f.write(" ".join(f"{v:.17e}" for v in mode) + "\n")
        for r in cov:
            f.write(" ".join(f"{v:.17e}" for v in r) + "\n")
    print(OUT, "sd:", np.sqrt(np.diag(cov)), "mode - true:", mode - eta0)


def load(path=OUT):
    """(mode [4], covariance [4][4]) of the stored approximation."""
    a = np.loadtxt(path)
    return a[0], a[1:5]


if __name__ == "__main__":
    main()
