"""Priors, random-walk Metropolis, delayed acceptance and chain statistics.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Posterior (Sec. 2, eq. (bayes)): mu^y(p) proportional to rho(y - G(p)) mu_0(p),
  i.e. log target = -Phi(p; y) + log mu_0(p); the normaliser is never needed.
* Algorithm 1 (one Metropolis-Hastings step) with a symmetric Gaussian random
  walk.  Each parameter moves in its own "step space": linear (eta = theta) or
  logarithmic (eta = log theta).  The target in eta-space carries the Jacobian
  d theta / d eta (= theta for log steps), so the chain samples the posterior
  over theta.  The paper's acceptance min(exp(Phi(x) - Phi(x_bar)), 1) is the
  special case of a flat prior; with a prior the prior ratio enters too.
* Priors: uniform on [lo, hi] (Sec. 3.1.2 Case 1) and log-normal with median m
  and log-standard-deviation s (Sec. 3.1.2 Case 3).
* Delayed acceptance (Christen & Fox 2005, not in the paper): a surrogate
  Phi~ screens each proposal; survivors get the exact Phi and a second test
  min(1, exp(Phi(x) - Phi(x_bar) + Phi~(x_bar) - Phi~(x))), which keeps the
  posterior exact for any surrogate.
* Algorithm 2 (the multi-proposal parallel Metropolis-Hastings step of
  Sec. 2.1, Calderhead 2014): N proposals, then the stationary distribution
  of the (N+1)-state chain A(i, j) = min(1, r(x^i, x^j)) / N (j != i),
  A(i, i) = 1 - sum_{j != i} A(i, j), r(x, y) = target(y) / target(x), and N
  draws from it.  Reading: the N proposals are drawn around an auxiliary
  point z ~ k(x_k, .) (as in the cited method), which makes the proposal of
  the N+1 points symmetric in them; drawn around x_k itself, as printed, the
  step would not leave the posterior invariant.
* Chain workflow of Sec. 2 / 2.1: discard a burn-in fraction, pool chains,
  report means and equal-tailed 95% credible intervals.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import ST_NONFINITE, ST_OUT_OF_SUPPORT, chain_randoms

PARAM_NAMES = ("a", "b", "d", "gamma", "r")


@dataclass
class Model:
    """Which of (a, b, d, gamma, r) are inferred, their priors and steps."""
    param_map: list            # indices into (a, b, d, gamma, r)
    fixed: np.ndarray          # [5] values used for the parameters not inferred
    prior_kind: list           # per inferred parameter: "uniform" | "lognormal"
    prior_p0: np.ndarray       # uniform: lower bound; lognormal: median
    prior_p1: np.ndarray       # uniform: upper bound; lognormal: sigma of log
    step_space: list           # per inferred parameter: "linear" | "log"
    step: np.ndarray           # random-walk standard deviation in step space
    chol: np.ndarray = None    # optional lower-triangular L: eta_bar = eta + L xi
    turing: bool = False       # also restrict (a, b, d) to the Turing space (Sec. 3.1.2 Case 2)
    poly_rho_T: float = None   # Example 1: also require the polynomial rho(t) > 0 on [0, T]
    extra: dict = field(default_factory=dict)

    @property
    def P(self):
        return len(self.param_map)

    def full_theta(self, theta):
        """[C][P] inferred values -> [C][8] (a, b, d, gamma, r, p1, p2, p3)."""
        theta = np.atleast_2d(theta)
        fixed = np.zeros(8)
        fixed[: len(self.fixed)] = self.fixed
        out = np.tile(fixed, (theta.shape[0], 1))
        for j, idx in enumerate(self.param_map):
            out[:, idx] = theta[:, j]
        return out

    def to_eta(self, theta):
        eta = np.array(theta, dtype=np.float64, copy=True)
        for j, sp in enumerate(self.step_space):
            if sp == "log":
                eta[:, j] = np.log(theta[:, j])
        return eta

    def to_theta(self, eta):
        th = np.array(eta, dtype=np.float64, copy=True)
        for j, sp in enumerate(self.step_space):
            if sp == "log":
                th[:, j] = np.exp(eta[:, j])
        return th

    def log_prior_eta(self, theta):
        """log mu_0(theta) + log |d theta / d eta| per chain; -inf outside the
        support.  Additive constants are dropped (they cancel in every
        acceptance ratio)."""
        theta = np.atleast_2d(theta)
        lp = np.zeros(theta.shape[0])
        for j in range(self.P):
            t = theta[:, j]
            with np.errstate(divide="ignore", invalid="ignore"):
                if self.prior_kind[j] == "uniform":
                    ok = (t >= self.prior_p0[j]) & (t <= self.prior_p1[j])
                    lpj = np.where(ok, 0.0, -np.inf)
                elif self.prior_kind[j] == "lognormal":
                    ok = t > 0
                    lt = np.log(np.where(ok, t, 1.0))
                    z = (lt - np.log(self.prior_p0[j])) / self.prior_p1[j]
                    lpj = np.where(ok, -lt - 0.5 * z * z, -np.inf)
                else:
                    raise ValueError(self.prior_kind[j])
                if self.step_space[j] == "log":
                    lpj = lpj + np.log(np.where(t > 0, t, 1.0))
            lp += lpj
        if self.turing:
            full = self.full_theta(theta)
            lp = np.where(in_turing_space(full[:, 0], full[:, 1], full[:, 2]), lp, -np.inf)
        if self.poly_rho_T is not None:
            from . import poly4_positive
            full = self.full_theta(theta)
            lp = np.where(poly4_positive(full[:, 5:8], self.poly_rho_T), lp, -np.inf)
        return lp


def in_turing_space(a, b, d):
    """The four inequalities of eq. (turing) for Schnakenberg kinetics at the
    homogeneous steady state (a + b, b / (a + b)^2): f_u + g_v < 0,
    f_u g_v - f_v g_u > 0, d f_u + g_v > 0, (d f_u + g_v)^2 - 4 d (f_u g_v -
    f_v g_u) > 0, with f_u = (b - a)/(b + a), g_v = -(a + b)^2 and
    f_u g_v - f_v g_u = (a + b)^2.  The uniform prior of Case 2 is uniform on
    this set (intersected with the box)."""
    a, b, d = (np.asarray(x, dtype=np.float64) for x in (a, b, d))
    with np.errstate(divide="ignore", invalid="ignore"):
        s = a + b
        fu = (b - a) / s
        gv = -s * s
        det = s * s
        c1 = fu + gv < 0
        c2 = det > 0
        c3 = d * fu + gv > 0
        c4 = (d * fu + gv) ** 2 - 4 * d * det > 0
    return c1 & c2 & c3 & c4 & (s > 0)


def _phi_of(phi_fn, model, theta, mask):
    """Phi at the rows of theta selected by mask; +inf and status elsewhere."""
    C = theta.shape[0]
    phi = np.full(C, np.inf)
    status = np.full(C, ST_OUT_OF_SUPPORT, dtype=np.uint32)
    idx = np.nonzero(mask)[0]
    if idx.size:
        ph, st = phi_fn(model.full_theta(theta[idx]))
        ph = np.asarray(ph, dtype=np.float64).copy()
        st = np.asarray(st, dtype=np.uint32)
        ph[st != 0] = np.inf
        phi[idx] = ph
        status[idx] = st
    return phi, status


class Chains:
    """C chains advanced in lock-step, one proposal per chain per step.

    ``phi_fn(theta_full [B][5]) -> (phi [B], status [B])`` is the forward solve
    plus log-likelihood; ``surrogate(theta [B][P]) -> phi_tilde [B]`` (optional)
    turns each step into a delayed-acceptance step.
    """

    def __init__(self, model: Model, theta0, seed: int, phi_fn, surrogate=None,
                 first_chain: int = 0):
        self.model = model
        self.theta = np.array(np.atleast_2d(theta0), dtype=np.float64)
        self.C = self.theta.shape[0]
        self.seed = int(seed)
        self.first_chain = int(first_chain)  # global index of chain 0 (sharded runs)
        self.phi_fn = phi_fn
        self.surrogate = surrogate
        self.step_index = 0
        self.lp = model.log_prior_eta(self.theta)
        self.phi, self.status = _phi_of(phi_fn, model, self.theta,
                                         np.isfinite(self.lp))
        self.phit = surrogate(self.theta) if surrogate is not None else None
        self.n_prop = 0
        self.n_pass1 = 0
        self.n_acc = 0
        self.n_solves = 0

    def step(self):
        """One step of Algorithm 1 (or its delayed-acceptance form)."""
        m = self.model
        xi, uu = chain_randoms(self.seed, self.C, self.step_index, self.first_chain)
        if m.chol is not None:  # correlated Gaussian random walk, increment L xi
            eta_bar = m.to_eta(self.theta) + xi[:, : m.P] @ np.asarray(m.chol).T
        else:
            eta_bar = m.to_eta(self.theta) + xi[:, : m.P] * np.asarray(m.step)[None, :]
        th_bar = m.to_theta(eta_bar)
        lp_bar = m.log_prior_eta(th_bar)
        in_support = np.isfinite(lp_bar)
        log_u1 = np.log(uu[:, 0])
        self.n_prop += self.C
        if self.surrogate is None:
            phi_bar, st_bar = _phi_of(self.phi_fn, m, th_bar, in_support)
            self.n_solves += int(in_support.sum())
            with np.errstate(invalid="ignore"):
                log_alpha = (-phi_bar + lp_bar) - (-self.phi + self.lp)
            accept = np.isfinite(phi_bar) & (log_u1 < log_alpha)
            phit_bar = None
        else:
            phit_bar = np.full(self.C, np.inf)
            if in_support.any():
                phit_bar[in_support] = self.surrogate(th_bar[in_support])
            with np.errstate(invalid="ignore"):
                log_a1 = (-phit_bar + lp_bar) - (-self.phit + self.lp)
            pass1 = in_support & (log_u1 < log_a1)
            self.n_pass1 += int(pass1.sum())
            phi_bar, st_bar = _phi_of(self.phi_fn, m, th_bar, pass1)
            self.n_solves += int(pass1.sum())
            log_u2 = np.log(uu[:, 1])
            with np.errstate(invalid="ignore"):
                log_a2 = (self.phi - phi_bar) + (phit_bar - self.phit)
            accept = pass1 & np.isfinite(phi_bar) & (log_u2 < log_a2)
        self.n_acc += int(accept.sum())
        self.theta[accept] = th_bar[accept]
        self.phi[accept] = phi_bar[accept]
        self.lp[accept] = lp_bar[accept]
        if phit_bar is not None:
            self.phit[accept] = phit_bar[accept]
        self.step_index += 1
        return accept

    def run(self, n_steps):
        """Runs n_steps; returns samples [n_steps][P][C] (state after each step)."""
        out = np.zeros((n_steps, self.model.P, self.C))
        for s in range(n_steps):
            self.step()
            out[s] = self.theta.T
        return out


def pmh_transition_matrix(log_target):
    """A of Algorithm 2 for the N+1 points with log target values log_target
    (-inf outside the support): A(i, j) = min(1, r(x^i, x^j)) / N for j != i,
    r(x^i, x^j) = exp(log_target[j] - log_target[i]), and the diagonal makes
    each row sum to 1."""
    lt = np.asarray(log_target, dtype=np.float64)
    n1 = lt.size
    N = n1 - 1
    A = np.zeros((n1, n1))
    for i in range(n1):
        for j in range(n1):
            if j == i:
                continue
            if lt[j] == -np.inf:
                r = 0.0
            elif lt[i] == -np.inf:
                r = np.inf
            else:
                with np.errstate(over="ignore"):  # exp -> inf, min(1, inf) = 1
                    r = np.exp(lt[j] - lt[i])
            A[i, j] = min(1.0, r) / N
        A[i, i] = 1.0 - A[i].sum()
    return A


def stationary(A):
    """The distribution pi with pi A = pi, sum(pi) = 1 (Algorithm 2 step 3):
    the linear system A^T pi - pi = 0 with its last equation replaced by the
    normalisation."""
    n1 = A.shape[0]
    M = A.T - np.eye(n1)
    M[-1, :] = 1.0
    rhs = np.zeros(n1)
    rhs[-1] = 1.0
    return np.linalg.solve(M, rhs)


class ParallelChains:
    """C independent chains advanced by Algorithm 2 with N proposals each;
    every step yields N samples per chain.  Random numbers of point t of a
    step (t = 0: the auxiliary point z; t = 1..N: the proposals) come from
    counters (first + chain, step, 0|1, t); the t-th of the N draws from the
    stationary distribution uses the uniform u_6 of point t."""

    def __init__(self, model: Model, theta0, seed: int, phi_fn, n_prop: int,
                 first_chain: int = 0):
        self.model = model
        self.theta = np.array(np.atleast_2d(theta0), dtype=np.float64)
        self.C = self.theta.shape[0]
        self.N = int(n_prop)
        self.seed = int(seed)
        self.first_chain = int(first_chain)
        self.phi_fn = phi_fn
        self.step_index = 0
        self.lp = model.log_prior_eta(self.theta)
        self.phi, _ = _phi_of(phi_fn, model, self.theta, np.isfinite(self.lp))
        self.n_prop = self.n_acc = self.n_solves = 0

    def _randoms(self, t):
        return chain_randoms(self.seed, self.C, self.step_index, self.first_chain, t)

    def _increment(self, xi):
        m = self.model
        if m.chol is not None:
            return xi[:, : m.P] @ np.asarray(m.chol).T
        return xi[:, : m.P] * np.asarray(m.step)[None, :]

    def step(self):
        """One step of Algorithm 2; returns the N new samples [N][P][C]."""
        m, C, N = self.model, self.C, self.N
        xi0, _ = self._randoms(0)
        eta_z = m.to_eta(self.theta) + self._increment(xi0)      # auxiliary point
        props = np.zeros((N, C, m.P))
        lps = np.zeros((N, C))
        u_draw = np.zeros((N, C))
        for t in range(1, N + 1):
            xi, uu = self._randoms(t)
            props[t - 1] = m.to_theta(eta_z + self._increment(xi))
            lps[t - 1] = m.log_prior_eta(props[t - 1])
            u_draw[t - 1] = uu[:, 0]
        flat = props.reshape(N * C, m.P)
        ok = np.isfinite(lps.reshape(-1))
        phis, _ = _phi_of(self.phi_fn, m, flat, ok)
        phis = phis.reshape(N, C)
        self.n_prop += N * C
        self.n_solves += int(ok.sum())
        out = np.zeros((N, m.P, C))
        for c in range(C):
            pts = np.concatenate([self.theta[c][None, :], props[:, c, :]], 0)
            phi_c = np.concatenate([[self.phi[c]], phis[:, c]])
            lp_c = np.concatenate([[self.lp[c]], lps[:, c]])
            with np.errstate(invalid="ignore"):
                lt = np.where(np.isfinite(phi_c) & np.isfinite(lp_c), -phi_c + lp_c, -np.inf)
            pi = stationary(pmh_transition_matrix(lt))
            cum = np.cumsum(pi)
            idx = [int(np.searchsorted(cum, u_draw[t, c] * cum[-1], side="right")) for t in range(N)]
            idx = [min(k, N) for k in idx]
            for t, k in enumerate(idx):
                out[t, :, c] = pts[k]
            self.n_acc += sum(1 for k in idx if k != 0)
            last = idx[-1]
            self.theta[c] = pts[last]
            self.phi[c] = phi_c[last]
            self.lp[c] = lp_c[last]
        self.step_index += 1
        return out

    def run(self, n_steps):
        """Runs n_steps; returns samples [n_steps * N][P][C]."""
        return np.concatenate([self.step() for _ in range(n_steps)], 0)


def summarize(samples, burn_frac=0.25):
    """Chain workflow of Sec. 2: drop a burn-in fraction of each chain, pool
    the chains, and report per-parameter mean and equal-tailed 95% credible
    interval.  samples: [steps][P][C]."""
    S = samples.shape[0]
    kept = samples[int(np.floor(burn_frac * S)):]
    pooled = kept.transpose(1, 0, 2).reshape(samples.shape[1], -1)
    return {
        "mean": pooled.mean(axis=1),
        "q025": np.quantile(pooled, 0.025, axis=1),
        "q975": np.quantile(pooled, 0.975, axis=1),
        "sd": pooled.std(axis=1, ddof=1),
    }


def ess_plain(x):
    """Effective sample size of one scalar chain from its definition,
    n / (1 + 2 sum_t rho_t), with the autocovariances rho_t summed in pairs
    until a pair sum turns negative (Geyer's initial positive sequence)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    xc = x - x.mean()
    var = np.dot(xc, xc) / n
    if var == 0:
        return float(n)
    def rho(t):
        return np.dot(xc[: n - t], xc[t:]) / n / var

    tau = -1.0  # 1 + 2 sum_{t>=1} rho_t written as -1 + 2 sum_{t>=0} rho_t
    t = 0
    while t + 1 < n:
        pair = rho(t) + rho(t + 1)
        if pair <= 0:
            break
        tau += 2.0 * pair
        t += 2
    return n / tau
