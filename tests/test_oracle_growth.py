"""The oracle's domain growth laws and Example 1's setting (Sec. 3.1.1):
the degree-4 polynomial with three degrees of freedom, the logistic law of
eq. (grates), their use in the time step, Example 1's initial state and the
stored datasets, each pinned against what the paper and the mathematics fix."""
import os

import numpy as np
import pytest

import oracle
import rd_synth
from oracle import mcmc, protocol

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TAYLOR = [0.6, 0.18, 0.036]  # exp(0.6 s) = 1 + 0.6 s + 0.18 s^2 + 0.036 s^3 + ...


def _th(p):
    return [0.1, 0.9, 10.0, 1000.0, 0.0] + list(p)


@pytest.mark.parametrize("p", [TAYLOR, [2.0, -3.0, 1.5], [0.0, 0.0, 0.0]])
def test_polynomial_meets_both_end_conditions(p):
    """rho(0) = 1 and rho(T) = rho_T for any p1, p2, p3: the coefficients of
    order 0 and 4 are the ones the two conditions fix."""
    T, rho_T = 600.0, 1.8
    assert oracle.growth("poly4", _th(p), 0.0, T, rho_T=rho_T)[0] == pytest.approx(1.0, abs=1e-15)
    assert oracle.growth("poly4", _th(p), T, T, rho_T=rho_T)[0] == pytest.approx(rho_T, rel=1e-14)


@pytest.mark.parametrize("kind,extra", [("poly4", dict(rho_T=1.8)),
                                        ("logistic", dict(logistic_K=np.exp(0.6))),
                                        ("exp", {})])
def test_growth_rate_is_the_derivative_of_rho(kind, extra):
    """rho'/rho against a central difference of rho (a wrong derivative or
    a dropped 1/T fails)."""
    theta = _th([1.1, -0.7, 0.4])
    theta[4] = 0.01 if kind == "logistic" else 0.002
    T = 600.0
    for t in (0.0 + 1.0, 150.0, 420.0, 599.0):
        rho, q = oracle.growth(kind, theta, t, T, **extra)
        rp = oracle.growth(kind, theta, t + 1e-3, T, **extra)[0]
        rm = oracle.growth(kind, theta, t - 1e-3, T, **extra)[0]
        assert q == pytest.approx((rp - rm) / 2e-3 / rho, rel=1e-6, abs=1e-12)


def test_logistic_law_solves_the_logistic_equation():
    """eq. (grates)' logistic law with the reading exp(0.6) for its printed
    constant: it solves rho' = lambda rho (1 - rho / K), rho(0) = 1 (checked
    against scipy's ODE integrator), and reaches about the exponential law's
    size e^0.6 at T = 600, as the paper states."""
    from scipy.integrate import solve_ivp
    lam, K = 0.01, np.exp(0.6)
    sol = solve_ivp(lambda t, r: lam * r * (1 - r / K), (0, 600), [1.0], rtol=1e-11,
                    atol=1e-13, dense_output=True)
    for t in (10.0, 100.0, 300.0, 600.0):
        assert oracle.growth("logistic", [0, 0, 0, 0, lam], t, 600.0, logistic_K=K)[0] == \
            pytest.approx(sol.sol(t)[0], rel=1e-8)
    rho_log = oracle.growth("logistic", [0, 0, 0, 0, lam], 600.0, 600.0, logistic_K=K)[0]
    assert abs(rho_log - np.exp(0.6)) < 0.01


def test_polynomial_with_taylor_coefficients_follows_the_exponential_law():
    """p = the cubic Taylor coefficients of exp(0.6 s) and rho_T = e^0.6 give a
    polynomial within 1e-3 of exp(0.001 t) on [0, 600]."""
    for t in np.linspace(0, 600, 13):
        r = oracle.growth("poly4", _th(TAYLOR), t, 600.0, rho_T=np.exp(0.6))[0]
        assert abs(r - np.exp(0.001 * t)) < 1e-3


def test_polynomial_support():
    """The growth prior's support: rho > 0 on the check grid."""
    assert oracle.poly4_positive(TAYLOR, np.exp(0.6))
    assert not oracle.poly4_positive([-3.0, 0.0, 0.0], 1.82)  # rho(0.5) < 0
    p = np.array([[0.6, 0.18, 0.036], [-3.0, 0.0, 0.0]])
    assert list(oracle.poly4_positive(p, 1.82)) == [True, False]
    m = mcmc.Model([5, 6, 7], np.zeros(5), ["uniform"] * 3, np.full(3, -20.0),
                   np.full(3, 20.0), ["linear"] * 3, np.full(3, 0.1), poly_rho_T=1.82)
    lp = m.log_prior_eta(p)
    assert np.isfinite(lp[0]) and lp[1] == -np.inf


@pytest.mark.parametrize("kind,theta,extra", [
    ("poly4", _th([1.1, -0.7, 0.4]), dict(rho_T=1.8)),
    ("logistic", [0.1, 0.9, 10.0, 0.0, 0.01], dict(logistic_K=np.exp(0.6)))])
def test_uniform_state_dilutes_by_the_growth_factor(kind, theta, extra):
    """gamma = 0, a uniform state c: no diffusion, and each semi-implicit step
    divides by 1 + tau m rho'/rho at t_n (m = 1), so the state after the run
    is c over the product of those factors, which tends to c / rho(T) as tau
    shrinks (rho'/rho integrates to log rho)."""
    n, c, T = 8, 1.3, 600.0
    th = list(theta)
    th[3] = 0.0
    for steps in (6000, 60000):
        tau = T / steps
        P = oracle.Problem(1, n, tau, steps, np.full(n, c), np.full(n, c), scheme="picard",
                           growth=kind, **extra)
        _, st, u, _ = P.forward(th)
        assert st == 0
        prod = np.prod([1.0 + tau * oracle.growth(kind, th, k * tau, T, **extra)[1]
                        for k in range(steps)])
        assert np.allclose(u, c / prod, rtol=1e-11)
        rho_end = oracle.growth(kind, th, T, T, **extra)[0]
        assert abs(u[0] * rho_end / c - 1.0) < 20.0 / steps


def test_cosine_mode_decays_with_the_time_dependent_factors():
    """gamma = 0: the cell-centred cosine mode k is an exact eigenvector, and
    each step multiplies it by 1 / (1 + tau m q_n + tau lambda_k / rho_n^2),
    with the polynomial law's rho_n and q_n."""
    n, k, steps, tau = 16, 3, 400, 1e-4
    T = steps * tau
    x = (np.arange(n) + 0.5) / n
    w0 = np.cos(np.pi * k * x)
    th = _th([1.1, -0.7, 0.4])
    th[3] = 0.0
    P = oracle.Problem(1, n, tau, steps, w0, w0, scheme="picard", growth="poly4", rho_T=1.8)
    _, st, u, _ = P.forward(th)
    lam = n * n * oracle.laplacian_eig(n, k)  # (4 / h^2) sin^2(pi k / 2n)
    fac = 1.0
    for s in range(steps):
        rho, q = oracle.growth("poly4", th, s * tau, T, rho_T=1.8)
        fac /= 1.0 + tau * q + tau * lam / rho**2
    assert 0.01 < fac < 0.5
    assert np.allclose(u, fac * w0, rtol=1e-10, atol=1e-14)


def test_example1_initial_state_and_datasets():
    """eq. (ic_gturing): both fields carry the same perturbation of the
    homogeneous steady state (1, 0.9) = (a + b, b / (a + b)^2) at a = 0.1,
    b = 0.9; the stored datasets start from it, and their noise level is 5 %
    of the range of u at T."""
    u0, v0 = protocol.example1_initial_state(100)
    assert np.allclose(u0 - 1.0, v0 - 0.9)
    assert oracle.steady_state(0.1, 0.9) == pytest.approx((1.0, 0.9))
    assert 0.0 < np.max(np.abs(u0 - 1.0)) <= 0.005 * 9
    for name in ("rd1d_e1_exp", "rd1d_e1_log"):
        spec = rd_synth.DATASETS[name]
        d = np.load(os.path.join(ROOT, "data", f"{name}.npz"))
        assert np.array_equal(d["u0"], u0) and np.array_equal(d["v0"], v0)
        clean = d["clean"][0]
        assert float(d["sigma"]) == pytest.approx(0.05 * (clean[0].max() - clean[0].min()))
        resid = (d["y"] - d["clean"]) / float(d["sigma"])
        assert abs(resid.std() - 1.0) < 0.15
        assert spec["n_steps"] * spec["tau"] == pytest.approx(600.0)
