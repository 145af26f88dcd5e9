"""Pins of the oracle's forward model against what the paper and the
mathematics fix (no GPU): known-answer RNG values, closed-form decay of
Laplacian eigenmodes, the steady state of Sec. 3.1.2, the Jacobian invariants
of eq. (turing), the continuum dispersion relation, brute-force dense solves
and library DCTs."""
import os

import numpy as np
import pytest
from scipy import stats
from scipy.fft import dct

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- RNG
def test_philox_known_answers():
    for row in _golden_rows("philox4x32_10_kat.txt"):
        vals = [int(x, 16) for x in row]
        out = oracle.philox4x32_10(vals[0:4], vals[4:6])
        assert [int(o) for o in out] == vals[6:10]


def test_chain_randoms_distribution():
    normals, uniforms = oracle.chain_randoms(seed=12345, n_chains=40000, step=7)
    assert np.all((uniforms > 0) & (uniforms < 1))
    assert stats.kstest(uniforms.ravel(), "uniform").pvalue > 1e-3
    assert stats.kstest(normals.ravel(), "norm").pvalue > 1e-3
    # distinct steps and seeds give distinct streams
    n2, _ = oracle.chain_randoms(seed=12345, n_chains=4, step=8)
    n3, _ = oracle.chain_randoms(seed=12346, n_chains=4, step=7)
    assert not np.allclose(normals[:4], n2) and not np.allclose(normals[:4], n3)


def test_chain_randoms_use_philox_words():
    """The uniforms are (w + 1/2) 2^-32 of the Philox words at counters
    (chain, step, 0|1, 0), key = (seed lo, seed hi)."""
    seed = (7 << 32) | 99
    _, uniforms = oracle.chain_randoms(seed=seed, n_chains=3, step=5)
    for c in range(3):
        w1 = oracle.philox4x32_10([c, 5, 1, 0], [99, 7])
        assert uniforms[c, 0] == (float(w1[2]) + 0.5) / 2**32
        assert uniforms[c, 1] == (float(w1[3]) + 0.5) / 2**32


# ---------------------------------------------------------------- solves
def _neumann_matrix_1d(n, alpha, beta_h):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = alpha
        for j in (i - 1, i + 1):
            jj = min(max(j, 0), n - 1)  # mirrored ghost value
            A[i, jj] -= beta_h
            A[i, i] += beta_h
    return A


@pytest.mark.parametrize("n", [1, 2, 3, 8, 64])
def test_thomas_matches_dense_solve(n):
    rng = np.random.default_rng(n)
    rhs = rng.standard_normal(n)
    alpha, beta_h = 1.3, 17.0
    A = _neumann_matrix_1d(n, alpha, beta_h)
    ref = np.linalg.solve(A, rhs)
    assert np.allclose(oracle.solve1d_thomas(alpha, beta_h, rhs), ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [4, 16, 96])
def test_dct_matrix_is_library_dct_and_neumann_eigenbasis(n):
    C = oracle.dct_matrix(n)
    x = np.random.default_rng(0).standard_normal(n)
    assert np.allclose(C @ x, dct(x, type=2, norm="ortho"), atol=1e-13)
    assert np.allclose(C @ C.T, np.eye(n), atol=1e-13)
    L = -_neumann_matrix_1d(n, 0.0, 1.0)  # stencil (w_{i-1} - 2 w_i + w_{i+1})
    for k in range(n):
        assert np.allclose(L @ C[k], -oracle.laplacian_eig(n, k) * C[k], atol=1e-12)


@pytest.mark.parametrize("n", [3, 8, 12])
def test_2d_dct_solve_matches_dense_solve(n):
    alpha, beta_h = 1.05, 9.0
    A1 = _neumann_matrix_1d(n, 0.0, beta_h)  # beta_h * (-Lap_1d)
    I = np.eye(n)
    A = alpha * np.eye(n * n) + np.kron(A1, I) + np.kron(I, A1)
    rhs = np.random.default_rng(3).standard_normal((n, n))
    ref = np.linalg.solve(A, rhs.ravel()).reshape(n, n)
    assert np.allclose(oracle.solve2d_dct(alpha, beta_h, rhs), ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("n", [16, 32])
def test_2d_dct_solve_matches_cg(n):
    rhs = 1.0 + np.random.default_rng(4).uniform(-0.5, 0.5, (n, n))
    alpha, beta_h = 1.0, 2.5e-4 * 10 * n * n
    x_cg, it = oracle.solve2d_cg(alpha, beta_h, rhs)
    assert it > 0
    assert np.allclose(oracle.solve2d_dct(alpha, beta_h, rhs), x_cg, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------- forward model
def test_table1_steady_state_constants():
    """Sec. 3.1.2: the constants of eq. (ic_numerical) are the homogeneous
    steady state at the Table 1 parameters."""
    for a, b, uc, vc in _golden_rows("table1_initial_state.txt"):
        us, vs = oracle.steady_state(float(a), float(b))
        assert round(us, 6) == float(uc)
        assert round(vs, 6) == float(vc)


@pytest.mark.parametrize("dim,n", [(1, 64), (2, 16)])
def test_steady_state_is_fixed(dim, n):
    """(a + b, b / (a + b)^2) is a fixed point of the kinetics and constants
    are in the kernel of the Neumann Laplacian, so the solution never moves.
    d = 1 keeps the state outside the Turing space (d f_u + g_v < 0), so
    roundoff is not amplified by an unstable mode; with d = 10 the fixed
    point is Turing-unstable and roundoff grows like exp(sigma t)."""
    a, b = 0.126779, 0.792366
    us, vs = oracle.steady_state(a, b)
    P = oracle.Problem(dim, n, 2.5e-4, 400, us, vs)
    _, st, u, v = P.forward([a, b, 1.0, 1000.0, 0.0])
    assert st == 0
    assert np.abs(u - us).max() < 1e-12 and np.abs(v - vs).max() < 1e-12
    _, st, u, v = P.forward([a, b, 10.0, 1000.0, 0.0])
    assert np.abs(u - us).max() < 1e-9 and np.abs(v - vs).max() < 1e-9


def _cos_mode(n, k):
    x = (np.arange(n) + 0.5) / n
    return np.cos(np.pi * k * x)


@pytest.mark.parametrize("r", [0.0, 0.05])
def test_cosine_mode_decay_1d_exact(r):
    """gamma = 0: cos(pi k x) on the cell-centred grid is an exact eigenvector;
    each step divides it by 1 + tau m r + tau D mu_k / (h^2 rho_n^2)."""
    n, k, tau, d, steps = 32, 3, 1e-3, 4.0, 50
    w0 = _cos_mode(n, k)
    P = oracle.Problem(1, n, tau, steps, w0, w0)
    _, st, u, v = P.forward([0.0, 0.0, d, 0.0, r])
    mu = 4 * np.sin(np.pi * k / (2 * n)) ** 2 * n * n
    fu = fv = 1.0
    for s in range(steps):
        rho2 = np.exp(2 * r * s * tau)
        fu /= 1 + tau * 1 * r + tau * mu / rho2
        fv /= 1 + tau * 1 * r + tau * d * mu / rho2
    assert np.allclose(u, fu * w0, rtol=1e-12, atol=1e-14)
    assert np.allclose(v, fv * w0, rtol=1e-12, atol=1e-14)


def test_cosine_mode_decay_2d_exact():
    n, k, l, tau, d, steps, r = 16, 2, 5, 5e-4, 3.0, 30, 0.02
    w0 = np.outer(_cos_mode(n, l), _cos_mode(n, k))
    P = oracle.Problem(2, n, tau, steps, w0, w0)
    _, st, u, v = P.forward([0.0, 0.0, d, 0.0, r])
    mu = (4 * np.sin(np.pi * k / (2 * n)) ** 2 + 4 * np.sin(np.pi * l / (2 * n)) ** 2) * n * n
    fu = fv = 1.0
    for s in range(steps):
        rho2 = np.exp(2 * r * s * tau)
        fu /= 1 + tau * 2 * r + tau * mu / rho2
        fv /= 1 + tau * 2 * r + tau * d * mu / rho2
    assert np.allclose(u, fu * w0, rtol=1e-11, atol=1e-14)
    assert np.allclose(v, fv * w0, rtol=1e-11, atol=1e-14)


def test_diffusion_converges_to_continuum_decay():
    """As h, tau -> 0 the decay of cos(pi k x) tends to exp(-D pi^2 k^2 t);
    the error falls with the first order in tau of backward Euler."""
    k, T, D = 2, 0.02, 1.0
    errs = []
    for n, steps in [(64, 50), (64, 100), (64, 200)]:
        w0 = _cos_mode(n, k)
        P = oracle.Problem(1, n, T / steps, steps, w0, w0)
        _, _, u, _ = P.forward([0.0, 0.0, D, 0.0, 0.0])
        amp = u @ w0 / (w0 @ w0)
        errs.append(abs(amp - np.exp(-D * np.pi**2 * k**2 * T)))
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]
    assert errs[2] < 2e-3


def _one_step_mode_matrix(a, b, d, g, n, k, tau, delta=1e-7):
    us, vs = oracle.steady_state(a, b)
    w = _cos_mode(n, k)
    cols = []
    for du, dv in [(1.0, 0.0), (0.0, 1.0)]:
        P = oracle.Problem(1, n, tau, 1, us + delta * du * w, vs + delta * dv * w)
        _, _, u, v = P.forward([a, b, d, g, 0.0])
        cols.append([(u - us) @ w / (w @ w) / delta, (v - vs) @ w / (w @ w) / delta])
    return np.array(cols).T


def test_reaction_jacobian_matches_turing_conditions():
    """Undo the implicit diffusion of one step of a single mode and recover the
    kinetics Jacobian J at the steady state; its trace and determinant must be
    the expressions printed in eq. (turing):
    f_u + g_v = (b - a)/(b + a) - (a + b)^2 and f_u g_v - f_v g_u = (a + b)^2."""
    a, b, d, g, n, k, tau = 0.1, 0.9, 10.0, 200.0, 64, 3, 1e-5
    A = _one_step_mode_matrix(a, b, d, g, n, k, tau)
    mu = 4 * np.sin(np.pi * k / (2 * n)) ** 2 * n * n
    M = np.diag([1 + tau * mu, 1 + tau * d * mu]) @ A
    J = (M - np.eye(2)) / (tau * g)
    assert np.trace(J) == pytest.approx((b - a) / (b + a) - (a + b) ** 2, rel=1e-5)
    assert np.linalg.det(J) == pytest.approx((a + b) ** 2, rel=1e-5)
    assert d * J[0, 0] + J[1, 1] == pytest.approx(d * (b - a) / (b + a) - (a + b) ** 2, rel=1e-5)


def test_growth_rate_matches_continuum_dispersion_relation():
    """Linear growth of a Turing-unstable mode: the per-step amplification of
    one mode tends to exp(sigma tau), sigma the larger root of the textbook
    dispersion relation sigma^2 - [gamma (f_u + g_v) - (1 + d) q^2] sigma
    + d q^4 - gamma (d f_u + g_v) q^2 + gamma^2 (a + b)^2 = 0 at q = pi k."""
    a, b, d, g = 0.1, 0.9, 10.0, 200.0
    fu, gv = (b - a) / (b + a), -(a + b) ** 2
    k, tau = 3, 2e-6
    q2 = (np.pi * k) ** 2
    tr = g * (fu + gv) - (1 + d) * q2
    det = d * q2**2 - g * (d * fu + gv) * q2 + g**2 * (a + b) ** 2
    sigma = 0.5 * (tr + np.sqrt(tr * tr - 4 * det))
    assert sigma > 0
    errs = []
    for n in (128, 256):
        A = _one_step_mode_matrix(a, b, d, g, n, k, tau)
        lam = np.max(np.linalg.eigvals(A).real)
        errs.append(abs(np.log(lam) / tau - sigma) / sigma)
    # second order in h: halving h cuts the error about four-fold
    assert errs[0] < 5e-3 and errs[1] < 0.35 * errs[0]


def test_loglik_closed_form():
    """Gaussian Phi of eq. (logl): from the steady state (which never moves),
    with y = u* + delta on every node, Phi = n_obs * N * delta^2 / (2 sigma^2)."""
    a, b = 0.1, 0.9
    us, vs = oracle.steady_state(a, b)
    n, delta, sigma = 16, 0.03, 0.01
    y = np.stack([np.full((n, n), us + delta), np.full((n, n), vs - delta)])[None]
    y = np.concatenate([y, y])  # two observation times
    P = oracle.Problem(2, n, 1e-3, 10, us, vs, y=y, obs_steps=[5, 10], field_mask=3, sigma=sigma)
    phi, st, _, _ = P.forward([a, b, 10.0, 200.0, 0.0])
    assert st == 0
    assert phi == pytest.approx(2 * 2 * n * n * delta**2 / (2 * sigma**2), rel=1e-10)
    # only v observed
    P = oracle.Problem(2, n, 1e-3, 10, us, vs, y=y[:1, 1:], obs_steps=[10], field_mask=2, sigma=sigma)
    phi, _, _, _ = P.forward([a, b, 10.0, 200.0, 0.0])
    assert phi == pytest.approx(n * n * delta**2 / (2 * sigma**2), rel=1e-10)


def test_divergent_solve_flags_nonfinite():
    """A parameter whose explicit reaction step is unstable must give status
    NONFINITE and Phi = +inf (the robust log-likelihood of Sec. 2)."""
    us, vs = oracle.steady_state(0.1, 0.9)
    n = 16
    P = oracle.Problem(2, n, 2.5e-4, 200, us + 0.1, vs, y=np.zeros((1, 1, n, n)),
                       obs_steps=[200], field_mask=1, sigma=0.01)
    phi, st, _, _ = P.forward([0.1, 0.9, 10.0, 5e4, 0.0])
    assert st & oracle.ST_NONFINITE and np.isinf(phi)


def test_batch_matches_single():
    ds = np.load(os.path.join(os.path.dirname(GOLDEN), "..", "data", "rd1d_n64.npz"))
    P = oracle.Problem(1, 64, 1e-4, 300, ds["u0"], ds["v0"], y=ds["clean"][:, :, :] * 0 + 1.0,
                       obs_steps=[300], field_mask=1, sigma=0.01)
    th = np.array([[0.1, 0.9, 10, 200, 0], [0.12, 0.8, 9, 180, 0], [0.1, 0.9, 10, 1e6, 0]])
    phi, st = P.forward_batch(th, n_threads=2)
    for i in range(3):
        p1, s1, _, _ = P.forward(th[i])
        assert s1 == st[i] and (phi[i] == p1 or (np.isinf(p1) and np.isinf(phi[i])))


# ---- the paper's semi-implicit scheme (Sec. 3.1.1, Example 1), 1-D --------

def _picard_pair(n, tau, steps, u0, v0, theta):
    out = {}
    for scheme in ("imex", "picard"):
        P = oracle.Problem(1, n, tau, steps, u0, v0, scheme=scheme)
        out[scheme] = P.forward(theta)[2:4]
    return out


def test_picard_keeps_the_steady_state_fixed():
    """(a + b, b/(a + b)^2) solves both linearised equations exactly:
    gamma (1 - u* v*) u* = gamma a and gamma u*^2 v* = gamma b."""
    a, b = 0.126779, 0.792366
    us, vs = oracle.steady_state(a, b)
    P = oracle.Problem(1, 16, 1e-4, 500, np.full(16, us), np.full(16, vs), scheme="picard")
    _, st, u, v = P.forward([a, b, 10.0, 1000.0, 0.0])
    assert st == 0
    assert np.max(np.abs(u - us)) < 1e-13 and np.max(np.abs(v - vs)) < 1e-13


def test_picard_equals_imex_without_reaction():
    """gamma = 0 leaves only the linear diffusion-dilution step, the same in
    both schemes, bit for bit."""
    rng = np.random.default_rng(4)
    u0, v0 = 1 + 0.01 * rng.standard_normal(32), 0.9 + 0.01 * rng.standard_normal(32)
    out = _picard_pair(32, 1e-3, 200, u0, v0, [0.1, 0.9, 10.0, 0.0, 0.02])
    assert np.array_equal(out["imex"][0], out["picard"][0])
    assert np.array_equal(out["imex"][1], out["picard"][1])


def test_dilution_of_a_uniform_state():
    """gamma = 0, uniform state c, growth r: each step divides by
    1 + tau m r (m = 1 in 1-D), in both schemes."""
    c, tau, r, steps = 1.3, 1e-3, 0.05, 300
    for scheme in ("imex", "picard"):
        P = oracle.Problem(1, 8, tau, steps, np.full(8, c), np.full(8, c), scheme=scheme)
        _, _, u, _ = P.forward([0.1, 0.9, 10.0, 0.0, r])
        assert np.allclose(u, c * (1 + tau * r) ** (-steps), rtol=1e-12)


def test_picard_and_imex_converge_together_at_first_order():
    """Both schemes are first order in tau and converge to the same
    solution: their difference at a fixed time halves with tau, and each
    one's distance to a fine-tau reference does too."""
    n, T = 32, 0.02
    x = (np.arange(n) + 0.5) / n
    u0 = 1.0 + 0.05 * np.cos(np.pi * x) + 0.02 * np.cos(3 * np.pi * x)
    v0 = 0.9 - 0.03 * np.cos(2 * np.pi * x)
    theta = [0.1, 0.9, 10.0, 200.0, 0.0]
    ref = _picard_pair(n, T / 2048, 2048, u0, v0, theta)["imex"][0]
    diffs, errs = [], []
    for k in (64, 128, 256):
        out = _picard_pair(n, T / k, k, u0, v0, theta)
        diffs.append(np.max(np.abs(out["picard"][0] - out["imex"][0])))
        errs.append(np.max(np.abs(out["picard"][0] - ref)))
    for d0, d1 in zip(diffs, diffs[1:]):
        assert 0.4 < d1 / d0 < 0.6
    for e0, e1 in zip(errs, errs[1:]):
        assert 0.35 < e1 / e0 < 0.65


# ---- the paper's semi-implicit scheme in 2-D (Sec. 3.1.1) ------------------

def _neumann_1d(n):
    """Unscaled 3-point Neumann Laplacian (ghost values mirror the boundary)."""
    L = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    L[0, 0] = L[-1, -1] = -1.0
    return L


@pytest.mark.parametrize("n", [4, 6, 8])
def test_2d_variable_diagonal_cg_matches_dense_solve(n):
    """[diag(alpha) - beta Lap_h] x = rhs, with alpha varying by node, against
    the dense 2-D operator built as a Kronecker sum (brute force)."""
    rng = np.random.default_rng(n)
    alpha = 1.0 + 0.3 * rng.random((n, n))
    rhs = rng.standard_normal((n, n))
    beta = 3.7
    L1 = _neumann_1d(n)
    A = np.diag(alpha.reshape(-1)) - beta * (np.kron(np.eye(n), L1) + np.kron(L1, np.eye(n)))
    ref = np.linalg.solve(A, rhs.reshape(-1)).reshape(n, n)
    x, it = oracle.solve2d_cg_var(alpha, beta, rhs)
    assert it > 0
    assert np.max(np.abs(x - ref)) < 1e-12 * np.max(np.abs(ref))


def test_picard_2d_keeps_the_steady_state_fixed():
    """As in 1-D: the homogeneous steady state solves both linearised 2-D
    equations exactly (to the CG tolerance)."""
    a, b = 0.126779, 0.792366
    us, vs = oracle.steady_state(a, b)
    n = 8
    P = oracle.Problem(2, n, 1e-4, 50, np.full((n, n), us), np.full((n, n), vs),
                       scheme="picard")
    _, st, u, v = P.forward([a, b, 10.0, 1000.0, 0.0])
    assert st == 0
    assert np.max(np.abs(u - us)) < 1e-12 and np.max(np.abs(v - vs)) < 1e-12


def test_picard_2d_equals_imex_without_reaction():
    """gamma = 0: both schemes take the same linear diffusion-dilution step
    (eigenbasis solve against CG, equal to the CG tolerance)."""
    n = 8
    rng = np.random.default_rng(5)
    u0 = 1 + 0.01 * rng.standard_normal((n, n))
    v0 = 0.9 + 0.01 * rng.standard_normal((n, n))
    out = {}
    for scheme in ("imex", "picard"):
        P = oracle.Problem(2, n, 1e-3, 40, u0, v0, scheme=scheme)
        out[scheme] = P.forward([0.1, 0.9, 10.0, 0.0, 0.02])[2:4]
    for f in range(2):
        assert np.max(np.abs(out["imex"][f] - out["picard"][f])) < 1e-12


def test_picard_2d_and_imex_converge_together_at_first_order():
    """Both 2-D schemes are first order in tau with the same limit: their
    difference at a fixed time halves with tau."""
    n, T = 8, 0.01
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    u0 = 1.0 + 0.05 * np.cos(np.pi * X) * np.cos(np.pi * Y) + 0.02 * np.cos(3 * np.pi * X)
    v0 = 0.9 - 0.03 * np.cos(2 * np.pi * Y)
    theta = [0.1, 0.9, 10.0, 200.0, 0.0]
    diffs = []
    for k in (32, 64, 128):
        out = {}
        for scheme in ("imex", "picard"):
            P = oracle.Problem(2, n, T / k, k, u0, v0, scheme=scheme)
            out[scheme] = P.forward(theta)[2]
        diffs.append(np.max(np.abs(out["picard"] - out["imex"])))
    for d0, d1 in zip(diffs, diffs[1:]):
        assert 0.4 < d1 / d0 < 0.6, diffs
