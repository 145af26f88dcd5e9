"""Pins of the oracle's sampler (no GPU): closed-form posteriors of a
linear-Gaussian toy, prior-only targets, delayed-acceptance exactness with a
deliberately poor surrogate, and the effective sample size of an AR(1) chain
whose integrated autocorrelation time is known in closed form."""
import numpy as np
import pytest

from oracle import mcmc


def _ess_pooled(samples):
    """Sum over chains of the per-chain ESS (for MCSE bounds in these tests)."""
    S, P, C = samples.shape
    return np.array([sum(mcmc.ess_plain(samples[:, p, c]) for c in range(C)) for p in range(P)])


def _toy_model(lo=-10.0, hi=10.0, step=(0.3, 0.3)):
    return mcmc.Model(param_map=[0, 1], fixed=np.zeros(5), prior_kind=["uniform"] * 2,
                      prior_p0=np.array([lo, lo]), prior_p1=np.array([hi, hi]),
                      step_space=["linear"] * 2, step=np.array(step))


A_TOY = np.array([[1.0, 0.5], [0.2, 1.5], [0.7, -0.4]])
Y_TOY = np.array([1.0, 2.0, 0.3])
SIG_TOY = 0.5


def _toy_phi(theta_full):
    th = theta_full[:, :2]
    r = Y_TOY[None, :] - th @ A_TOY.T
    return (r * r).sum(1) / (2 * SIG_TOY**2), np.zeros(th.shape[0], np.uint32)


def _toy_posterior():
    prec = A_TOY.T @ A_TOY / SIG_TOY**2
    cov = np.linalg.inv(prec)
    mean = cov @ (A_TOY.T @ Y_TOY) / SIG_TOY**2
    return mean, cov


def _check_gaussian(samples, mean, cov, burn=200):
    kept = samples[burn:]
    ess = _ess_pooled(kept)
    pooled = kept.transpose(1, 0, 2).reshape(2, -1)
    sd = np.sqrt(np.diag(cov))
    mcse = sd / np.sqrt(ess)
    assert np.all(np.abs(pooled.mean(1) - mean) < 3.5 * mcse), (pooled.mean(1), mean, mcse)
    # variance: MCSE of a Gaussian variance estimate ~ var * sqrt(2 / ess)
    var = pooled.var(1, ddof=1)
    assert np.all(np.abs(var - sd**2) < 3.5 * sd**2 * np.sqrt(2 / ess)), (var, sd**2)


def test_linear_gaussian_posterior():
    """G(theta) = A theta with Gaussian noise and a flat (very wide uniform)
    prior: the posterior is N((A'A)^-1 A'y, sigma^2 (A'A)^-1)."""
    mean, cov = _toy_posterior()
    m = _toy_model()
    ch = mcmc.Chains(m, np.tile(mean, (32, 1)) + 0.1, seed=3, phi_fn=_toy_phi)
    samples = ch.run(1500)
    _check_gaussian(samples, mean, cov)
    assert 0.2 < ch.n_acc / ch.n_prop < 0.9


def test_delayed_acceptance_is_exact_with_poor_surrogate():
    """Christen-Fox exactness: a surrogate that is wrong (scaled, shifted and
    tilted) still leaves the posterior unchanged."""
    mean, cov = _toy_posterior()
    m = _toy_model()

    def bad_surrogate(theta):
        phi, _ = _toy_phi(m.full_theta(theta))
        return 0.6 * phi + 3.0 * theta[:, 0] - 7.0

    ch = mcmc.Chains(m, np.tile(mean, (32, 1)) - 0.1, seed=5, phi_fn=_toy_phi,
                     surrogate=bad_surrogate)
    samples = ch.run(1500)
    _check_gaussian(samples, mean, cov)
    assert ch.n_solves == ch.n_pass1 < ch.n_prop


def test_uniform_prior_flat_likelihood():
    """Phi = 0 with a uniform prior on [0, 1] x [0, 2]: samples are uniform
    (mean at the centre, variance (hi - lo)^2 / 12)."""
    m = mcmc.Model(param_map=[0, 1], fixed=np.zeros(5), prior_kind=["uniform"] * 2,
                   prior_p0=np.array([0.0, 0.0]), prior_p1=np.array([1.0, 2.0]),
                   step_space=["linear"] * 2, step=np.array([0.3, 0.6]))
    flat = lambda th: (np.zeros(th.shape[0]), np.zeros(th.shape[0], np.uint32))
    ch = mcmc.Chains(m, np.tile([0.5, 1.0], (32, 1)), seed=9, phi_fn=flat)
    s = ch.run(1500)[100:]
    ess = _ess_pooled(s)
    pooled = s.transpose(1, 0, 2).reshape(2, -1)
    sd = np.array([1.0, 2.0]) / np.sqrt(12)
    assert np.all(np.abs(pooled.mean(1) - [0.5, 1.0]) < 3.5 * sd / np.sqrt(ess))
    assert np.all((pooled >= [[0.0], [0.0]]) & (pooled <= [[1.0], [2.0]]))
    assert np.allclose(pooled.var(1), sd**2, rtol=0.1)


def test_lognormal_prior_in_log_space():
    """Phi = 0, log-normal prior (median m, sigma s), random walk in log theta:
    log theta ~ N(log m, s^2)."""
    med, sig = np.array([10.0, 200.0]), np.array([0.5, 0.5])
    m = mcmc.Model(param_map=[2, 3], fixed=np.array([0.1, 0.9, 0, 0, 0]),
                   prior_kind=["lognormal"] * 2, prior_p0=med, prior_p1=sig,
                   step_space=["log"] * 2, step=np.array([0.6, 0.6]))
    flat = lambda th: (np.zeros(th.shape[0]), np.zeros(th.shape[0], np.uint32))
    ch = mcmc.Chains(m, np.tile(med, (32, 1)), seed=11, phi_fn=flat)
    s = np.log(ch.run(1500)[100:])
    ess = _ess_pooled(s)
    pooled = s.transpose(1, 0, 2).reshape(2, -1)
    assert np.all(np.abs(pooled.mean(1) - np.log(med)) < 3.5 * sig / np.sqrt(ess))
    assert np.allclose(pooled.std(1), sig, rtol=0.08)


def test_lognormal_prior_with_linear_steps():
    """The same log-normal target sampled with steps in theta itself (the
    prior density then carries its 1/theta factor): log theta ~ N(log m, s^2)."""
    med, sig = np.array([2.0]), np.array([0.3])
    m = mcmc.Model(param_map=[2], fixed=np.array([0.1, 0.9, 0, 200, 0]),
                   prior_kind=["lognormal"], prior_p0=med, prior_p1=sig,
                   step_space=["linear"], step=np.array([1.0]))
    flat = lambda th: (np.zeros(th.shape[0]), np.zeros(th.shape[0], np.uint32))
    ch = mcmc.Chains(m, np.tile(med, (32, 1)), seed=12, phi_fn=flat)
    s = np.log(ch.run(2000)[100:])
    ess = _ess_pooled(s)
    pooled = s.reshape(-1)
    assert abs(pooled.mean() - np.log(2.0)) < 3.5 * 0.3 / np.sqrt(ess[0])
    assert pooled.std() == pytest.approx(0.3, rel=0.08)


def test_rejects_outside_support_and_nonfinite():
    m = _toy_model(lo=0.0, hi=1.0, step=(5.0, 5.0))
    calls = []

    def phi_fn(th):
        calls.append(th.copy())
        return np.zeros(th.shape[0]), np.zeros(th.shape[0], np.uint32)

    ch = mcmc.Chains(m, np.tile([0.5, 0.5], (64, 1)), seed=1, phi_fn=phi_fn)
    s = ch.run(20)
    evaluated = np.concatenate(calls[1:])[:, :2]
    assert np.all((evaluated >= 0) & (evaluated <= 1))  # no solve outside support
    assert np.all((s >= 0) & (s <= 1))

    def nan_fn(th):
        return np.full(th.shape[0], np.nan), np.full(th.shape[0], 2, np.uint32)

    m2 = _toy_model()
    ch2 = mcmc.Chains(m2, np.tile([0.5, 0.5], (8, 1)), seed=1, phi_fn=_toy_phi)
    ch2.phi_fn = nan_fn
    before = ch2.theta.copy()
    ch2.run(10)
    assert np.array_equal(ch2.theta, before)


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.9])
def test_ess_of_ar1(phi):
    """AR(1) x_t = phi x_{t-1} + e_t has integrated autocorrelation time
    (1 + phi) / (1 - phi), so ESS = n (1 - phi) / (1 + phi)."""
    rng = np.random.default_rng(int(phi * 10))
    n, reps = 20000, 8
    vals = []
    for _ in range(reps):
        e = rng.standard_normal(n)
        x = np.empty(n)
        x[0] = e[0] / np.sqrt(1 - phi**2)
        for t in range(1, n):
            x[t] = phi * x[t - 1] + e[t]
        vals.append(mcmc.ess_plain(x))
    expect = n * (1 - phi) / (1 + phi)
    assert np.mean(vals) == pytest.approx(expect, rel=0.1)


def test_summarize_credible_interval():
    rng = np.random.default_rng(0)
    s = rng.standard_normal((4000, 1, 8))
    out = mcmc.summarize(s, burn_frac=0.25)
    assert out["q025"][0] == pytest.approx(-1.96, abs=0.05)
    assert out["q975"][0] == pytest.approx(1.96, abs=0.05)
    assert abs(out["mean"][0]) < 0.03


def test_correlated_proposal_keeps_posterior():
    """A lower-triangular proposal factor L (increment L xi) is still a
    symmetric random walk: the linear-Gaussian posterior is unchanged."""
    mean, cov = _toy_posterior()
    m = _toy_model()
    m.chol = np.linalg.cholesky(2.38**2 / 2 * cov)
    ch = mcmc.Chains(m, np.tile(mean, (32, 1)) + 0.1, seed=13, phi_fn=_toy_phi)
    samples = ch.run(1500)
    _check_gaussian(samples, mean, cov)
    assert 0.2 < ch.n_acc / ch.n_prop < 0.6


def test_pmh_stationary_is_the_normalised_target():
    """Algorithm 2's (N+1)-state chain: A is row-stochastic and non-negative,
    and by detailed balance (min(1, t_j/t_i) t_i is symmetric) its stationary
    distribution is the target restricted to the points, normalised; points
    outside the support get 0."""
    rng = np.random.default_rng(3)
    for N in (1, 2, 4, 8, 16):
        lt = rng.normal(0.0, 3.0, N + 1)
        if N >= 4:
            lt[2] = -np.inf
        A = mcmc.pmh_transition_matrix(lt)
        assert np.all(A >= -1e-15) and np.allclose(A.sum(1), 1.0, atol=1e-14)
        pi = mcmc.stationary(A)
        w = np.exp(lt - lt.max())
        assert np.allclose(pi, w / w.sum(), rtol=1e-10, atol=1e-14)
        assert np.allclose(pi @ A, pi, atol=1e-14)


def test_pmh_linear_gaussian_posterior():
    """Algorithm 2 (N = 4 proposals around an auxiliary point) samples the
    closed-form linear-Gaussian posterior."""
    mean, cov = _toy_posterior()
    m = _toy_model(step=(0.25, 0.25))
    ch = mcmc.ParallelChains(m, np.tile(mean, (16, 1)) + 0.1, 21, _toy_phi, n_prop=4)
    samples = ch.run(500)  # [2000][P][16]
    _check_gaussian(samples, mean, cov, burn=200)
    assert 0 < ch.n_acc < ch.n_prop


def test_pmh_reading_auxiliary_point_is_needed():
    """The reading behind Algorithm 2's proposals: drawn around x_k itself (as
    printed) the step is not invariant -- with 8 proposals of a wide step it
    visibly shrinks the posterior variance -- while drawn around an auxiliary
    point z ~ k(x_k, .) it is not."""
    mean, cov = _toy_posterior()
    m = _toy_model(step=(0.6, 0.6))

    class Printed(mcmc.ParallelChains):
        def _randoms(self, t):
            xi, uu = super()._randoms(t)
            return (xi * 0.0 if t == 0 else xi), uu  # z = x_k

    ratios = {}
    for cls in (mcmc.ParallelChains, Printed):
        s = cls(m, np.tile(mean, (32, 1)), 5, _toy_phi, n_prop=8).run(400)[800:]
        pooled = s.transpose(1, 0, 2).reshape(2, -1)
        ratios[cls] = pooled.var(1) / np.diag(cov)
    assert np.all(np.abs(ratios[mcmc.ParallelChains] - 1.0) < 0.06)
    assert np.all(ratios[Printed] < 0.92)


def _unstable_by_dispersion(a, b, d):
    """Brute force: the homogeneous state is stable without diffusion and some
    wavenumber k^2 > 0 grows under diffusion, from the eigenvalues of
    J - k^2 diag(1, d) (J = the Schnakenberg Jacobian at (a + b, b/(a+b)^2))."""
    s = a + b
    J = np.array([[(b - a) / s, s * s], [-2 * b / s, -s * s]])
    if np.max(np.linalg.eigvals(J).real) >= 0:
        return False
    ks = np.concatenate([np.linspace(1e-6, 5, 4001), np.geomspace(5, 1e4, 2000)])
    return any(np.max(np.linalg.eigvals(J - k2 * np.diag([1.0, d])).real) > 0 for k2 in ks)


def test_turing_space_matches_the_dispersion_relation():
    """eq. (turing) against the linear stability of the reaction-diffusion
    system checked wavenumber by wavenumber."""
    assert mcmc.in_turing_space(0.1, 0.9, 10.0)
    assert not mcmc.in_turing_space(0.1, 0.9, 1.0)   # equal diffusion: no patterns
    rng = np.random.default_rng(11)
    pts = np.column_stack([rng.uniform(0, 1, 300), rng.uniform(0, 2, 300),
                           rng.uniform(1, 40, 300)])
    inside = mcmc.in_turing_space(pts[:, 0], pts[:, 1], pts[:, 2])
    assert 0.1 < inside.mean() < 0.9
    for (a, b, d), ins in zip(pts, inside):
        assert ins == _unstable_by_dispersion(a, b, d), (a, b, d)


def test_turing_prior_rejects_outside():
    m = mcmc.Model(param_map=[0, 1], fixed=np.array([0.1, 0.9, 10.0, 200.0, 0.0]),
                   prior_kind=["uniform"] * 2, prior_p0=np.array([0.0, 0.0]),
                   prior_p1=np.array([1.0, 2.0]), step_space=["linear"] * 2,
                   step=np.array([0.1, 0.1]), turing=True)
    lp = m.log_prior_eta(np.array([[0.1, 0.9], [0.9, 0.1], [0.5, 1.9]]))
    assert lp[0] == 0.0 and lp[1] == -np.inf
    assert (lp[2] == 0.0) == bool(mcmc.in_turing_space(0.5, 1.9, 10.0))
