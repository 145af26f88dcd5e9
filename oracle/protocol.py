"""The paper's data protocol for steady-state measurements (Sec. 3.1.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): generates synthetic
data with the FP64 oracle; nothing here runs on the GPU path.

* Initial state of eq. (ic_numerical): the homogeneous steady state
  (a + b, b / (a + b)^2) plus 0.0016 cos(2 pi (x + y)) + 0.01 sum_{j=1..8}
  cos(2 pi j x) in both fields (in 1-D the y terms are dropped).
* Evolve until the L2 norm of the discrete time derivative,
  (h^dim sum over both fields of ((w^{n+1} - w^n) / tau)^2)^(1/2), falls below
  a threshold (1e-5 in the paper); the time reached is T.  Continue to 2T and
  accept the state at T as stationary if the L2 norm of w(2T) - w(T) is below
  the threshold too.
* Measurement: the stationary field plus Gaussian noise whose standard
  deviation is a fraction (5 % or 10 %) of the field's range.
* Example 1's initial state, eq. (ic_gturing).
"""
from __future__ import annotations

import numpy as np

from . import Problem, steady_state


def paper_initial_state(dim, n, a, b):
    """Initial state of eq. (ic_numerical) on the cell-centred grid
    x_i = (i + 1/2) / n; returns (u0, v0)."""
    x = (np.arange(n) + 0.5) / n
    us, vs = steady_state(a, b)
    if dim == 1:
        pert = 0.0016 * np.cos(2 * np.pi * x) + 0.01 * sum(
            np.cos(2 * np.pi * j * x) for j in range(1, 9))
    else:
        X, Y = x[None, :], x[:, None]  # [y][x]
        pert = 0.0016 * np.cos(2 * np.pi * (X + Y)) + 0.01 * sum(
            np.cos(2 * np.pi * j * X) for j in range(1, 9))
    return us + pert, vs + pert


def example1_initial_state(n):
    """Initial state of eq. (ic_gturing) (Example 1) on the cell-centred grid
    x_i = (i + 1/2) / n of the unit interval: the homogeneous steady state
    (1, 0.9) of a = 0.1, b = 0.9 plus 0.005 sum_{k=1..9} sin(k pi x) in both
    fields; returns (u0, v0)."""
    x = (np.arange(n) + 0.5) / n
    pert = 0.005 * sum(np.sin(k * np.pi * x) for k in range(1, 10))
    return 1.0 + pert, 0.9 + pert


def _l2(w, h, dim):
    return float(np.sqrt(h**dim * np.sum(w * w)))


def evolve_to_steady_state(dim, n, tau, theta, u0, v0, threshold=1e-5, max_steps=1_000_000,
                           chunk=1):
    """Runs the IMEX scheme from (u0, v0) on a fixed domain one step at a time
    until the discrete time derivative's L2 norm is below threshold, then as
    many steps again.  Returns dict(u, v, steps_T, T, dwdt, diff_2T,
    stationary)."""
    h = 1.0 / n
    u, v = np.array(u0, dtype=np.float64), np.array(v0, dtype=np.float64)
    theta = list(theta) + [0.0] * (5 - len(theta))
    theta[4] = 0.0  # fixed domain
    steps = 0
    dwdt = np.inf
    while steps < max_steps:
        _, st, u1, v1 = Problem(dim, n, tau, chunk, u, v).forward(theta)
        if st != 0:
            raise RuntimeError(f"solve failed with status {st}")
        dwdt = _l2(np.concatenate([(u1 - u).ravel(), (v1 - v).ravel()]) / (tau * chunk), h, dim)
        u, v = u1, v1
        steps += chunk
        if dwdt < threshold:
            break
    else:
        raise RuntimeError("no steady state within max_steps")
    _, st, u2, v2 = Problem(dim, n, tau, steps, u, v).forward(theta)
    diff = _l2(np.concatenate([(u2 - u).ravel(), (v2 - v).ravel()]), h, dim)
    return dict(u=u, v=v, steps_T=steps, T=steps * tau, dwdt=dwdt, diff_2T=diff,
                stationary=diff < threshold)


def range_noise(w, fraction, rng):
    """w + N(0, (fraction * (max w - min w))^2) noise; returns (y, sigma)."""
    sigma = fraction * float(np.max(w) - np.min(w))
    return w + rng.normal(0.0, sigma, np.shape(w)), sigma
