"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds only random draws and the recipe (sizes, seeds) of the
synthetic workloads; it contains none of the method's arithmetic.  The paper
uses computer-generated patterns as data (Sec. 1.2, Sec. 3.1.2), so every
workload here is synthetic: a known initial state (the homogeneous steady state
of the true parameters plus seeded uniform noise), observations of the solution
at the true parameters plus seeded Gaussian noise, seeded chain starts and
seeded prior draws.
"""
from __future__ import annotations

import numpy as np

TRUE_THETA = (0.1, 0.9, 10.0, 200.0)  # (a, b, d, gamma)

# name -> recipe.  dims/sizes/steps follow the five workloads: the 1-D FP64
# case, the 2-D fixed-domain cases at 64^2/96^2/128^2 and the growing domain.
DATASETS = {
    "rd1d_n64": dict(dim=1, n=64, tau=1e-4, n_steps=10000, theta=(0.1, 0.9, 10.0, 200.0, 0.0),
                     obs_frac=(1.0,), field_mask=1, sigma=0.01, ic_amp=0.01,
                     ic_seed=0, obs_seed=1, dtype="f64"),
    "rd2d_n64": dict(dim=2, n=64, tau=2.5e-4, n_steps=8000, theta=(0.1, 0.9, 10.0, 200.0, 0.0),
                     obs_frac=(1.0,), field_mask=3, sigma=0.01, ic_amp=0.01,
                     ic_seed=10, obs_seed=11, dtype="f32"),
    "rd2d_n96": dict(dim=2, n=96, tau=2.5e-4, n_steps=8000, theta=(0.1, 0.9, 10.0, 200.0, 0.0),
                     obs_frac=(1.0,), field_mask=3, sigma=0.01, ic_amp=0.01,
                     ic_seed=20, obs_seed=21, dtype="f32"),
    "rd2d_n128": dict(dim=2, n=128, tau=2.5e-4, n_steps=8000, theta=(0.1, 0.9, 10.0, 200.0, 0.0),
                      obs_frac=(1.0,), field_mask=3, sigma=0.01, ic_amp=0.01,
                      ic_seed=30, obs_seed=31, dtype="f32"),
    "rd2d_n128_grow": dict(dim=2, n=128, tau=1e-4, n_steps=50000,
                           theta=(0.1, 0.9, 10.0, 200.0, 0.01),
                           obs_frac=(0.2, 0.4, 0.6, 0.8, 1.0), field_mask=1, sigma=0.02,
                           ic_amp=0.01, ic_seed=40, obs_seed=41, dtype="f32"),
    # Example 1 (Sec. 3.1.1): 1-D growing interval, fixed kinetics, the paper's
    # semi-implicit scheme, h = 1e-2, tau = 1e-4, T = 600; data from the
    # exponential law exp(0.001 t) or the logistic law (rate 0.01, capacity
    # exp(0.6)); the initial state of eq. (ic_gturing); u and v observed at T
    # with noise of 5 % of the range of u
    "rd1d_e1_exp": dict(dim=1, n=100, tau=1e-4, n_steps=6_000_000,
                        theta=(0.1, 0.9, 10.0, 1000.0, 0.001), growth="exp",
                        logistic_K=1.0, scheme="picard", ic="example1",
                        obs_frac=(1.0,), field_mask=3, noise_frac=0.05, obs_seed=51,
                        dtype="f64"),
    "rd1d_e1_log": dict(dim=1, n=100, tau=1e-4, n_steps=6_000_000,
                        theta=(0.1, 0.9, 10.0, 1000.0, 0.01), growth="logistic",
                        logistic_K=float(np.exp(0.6)), scheme="picard", ic="example1",
                        obs_frac=(1.0,), field_mask=3, noise_frac=0.05, obs_seed=52,
                        dtype="f64"),
}


def obs_steps(spec):
    """Observation step indices: equally spaced fractions of the final time."""
    return [int(round(f * spec["n_steps"])) for f in spec["obs_frac"]]


def uniform_noise(shape, seed, amp):
    """U(-amp, amp) per node, seeded."""
    return np.random.default_rng(seed).uniform(-amp, amp, size=shape)


def gaussian_noise(shape, seed, sigma):
    """N(0, sigma^2) per node, seeded."""
    return np.random.default_rng(seed).normal(0.0, sigma, size=shape)


def chain_starts(center, n_chains, seed, rel=0.01):
    """Chain starting points center * exp(rel * N(0, 1)), seeded, [C][P]."""
    center = np.asarray(center, dtype=np.float64)
    z = np.random.default_rng(seed).standard_normal((n_chains, center.size))
    return center[None, :] * np.exp(rel * z)


def lognormal_draws(medians, sigmas, n, seed):
    """n draws median * exp(sigma * N(0, 1)) per coordinate, seeded, [n][P]."""
    medians = np.asarray(medians, dtype=np.float64)
    sigmas = np.asarray(sigmas, dtype=np.float64)
    z = np.random.default_rng(seed).standard_normal((n, medians.size))
    return medians[None, :] * np.exp(sigmas[None, :] * z)


def uniform_draws(lo, hi, n, seed):
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return np.random.default_rng(seed).uniform(lo, hi, size=(n, lo.size))
