"""The steady-state data protocol of Sec. 3.1.2 in the oracle: the initial
state of eq. (ic_numerical), evolution until the discrete time derivative's
L2 norm is below the threshold with the 2T confirmation, and noise relative
to the solution's range."""
import os

import numpy as np

from oracle import protocol

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_initial_state.txt")


def test_initial_state_means_are_the_printed_constants():
    """The cosine terms of eq. (ic_numerical) average to zero on the
    cell-centred grid, so the field means are the printed constants
    (0.919145, 0.937903) at the Table 1 parameters."""
    a, b, uc, vc = np.loadtxt(GOLDEN)
    for dim, n in ((1, 64), (2, 32), (2, 128)):
        u0, v0 = protocol.paper_initial_state(dim, n, a, b)
        assert u0.shape == ((n,) if dim == 1 else (n, n))
        assert abs(u0.mean() - uc) < 5e-7 and abs(v0.mean() - vc) < 5e-7
        assert np.allclose(u0 - u0.mean(), v0 - v0.mean())  # the same perturbation
        assert 0.07 < u0.max() - u0.min() < 0.2


def test_pure_diffusion_reaches_the_mean():
    """gamma = 0: the steady state of the Neumann heat equation is the mean of
    the initial state; the protocol stops near it and confirms it at 2T."""
    u0, v0 = protocol.paper_initial_state(1, 32, 0.1, 0.9)
    out = protocol.evolve_to_steady_state(1, 32, 1e-3, [0.1, 0.9, 10.0, 0.0], u0, v0)
    assert out["dwdt"] < 1e-5 and out["stationary"]
    # the slowest mode decays at rate pi^2 (k = 1, D = 1): |u - mean| ~ dwdt / pi^2
    assert np.max(np.abs(out["u"] - u0.mean())) < 1e-5
    assert np.max(np.abs(out["v"] - v0.mean())) < 1e-5


def test_schnakenberg_pattern_is_stationary():
    """The Turing pattern of the 1-D system at Table 1's (a, b), d = 10,
    gamma = 200: the protocol terminates, the 2T check passes, and one more
    step barely moves the state."""
    a, b, _, _ = np.loadtxt(GOLDEN)
    u0, v0 = protocol.paper_initial_state(1, 32, a, b)
    out = protocol.evolve_to_steady_state(1, 32, 1e-4, [a, b, 10.0, 200.0], u0, v0)
    assert out["stationary"] and out["dwdt"] < 1e-5
    assert out["u"].max() - out["u"].min() > 0.1  # a pattern, not the homogeneous state


def test_range_relative_noise():
    rng = np.random.default_rng(5)
    w = np.linspace(0.5, 2.5, 40000)
    for frac in (0.05, 0.10):
        y, sigma = protocol.range_noise(w, frac, rng)
        assert sigma == frac * 2.0
        assert abs(np.std(y - w) / sigma - 1.0) < 0.02
