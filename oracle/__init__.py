"""FP64 CPU oracle for the Bayesian identification of Schnakenberg parameters.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1605_04718_gb300`` and never imports it.

Contents (each function cites the part of arXiv:1605.04718 it follows):

* ``rd_oracle.c`` -- Philox4x32-10, the IMEX forward solve of eq.
  (schnakenberg)/(reactions) with the Neumann finite-difference Laplacian of
  Sec. 3.1.1, the implicit solves (Thomas in 1-D; eigenbasis diagonalisation
  and plain CG in 2-D) and the Gaussian log-likelihood of eq. (logl);
* ``mcmc.py`` -- priors, random-walk Metropolis (Algorithm 1), delayed
  acceptance with a surrogate, and the chain post-processing of Sec. 2 / 2.1;
* ``mlp.py`` -- the surrogate network in FP64 (forward, backward, Adam);
* ``make_datasets.py`` -- writes the synthetic observation datasets.

Parity status of each function is listed in its docstring; every function here
is pinned by a ``-m "not gpu"`` test against closed forms, brute force, a
library routine or a published known-answer value.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librd_oracle.so")
_lib = None

ST_OUT_OF_SUPPORT = 1
ST_NONFINITE = 2
ST_NOT_CONVERGED = 4


def build(force: bool = False) -> str:
    """Compile the C oracle with the host gcc (no CPU-specific flags, no FMA
    contraction, so x86-64 and aarch64 hosts give the same arithmetic)."""
    src = os.path.join(_HERE, "rd_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call([
        "gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
        "-o", tmp, src, "-lm", "-lpthread"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int), ("n_steps", ctypes.c_int),
        ("tau", ctypes.c_double), ("m_growth", ctypes.c_int),
        ("n_obs", ctypes.c_int), ("obs_steps", ctypes.POINTER(ctypes.c_int)),
        ("field_mask", ctypes.c_int), ("y", ctypes.POINTER(ctypes.c_double)),
        ("sigma", ctypes.c_double), ("u0", ctypes.POINTER(ctypes.c_double)),
        ("v0", ctypes.POINTER(ctypes.c_double)), ("w_max", ctypes.c_double),
        ("solver", ctypes.c_int), ("scheme", ctypes.c_int),
        ("growth_kind", ctypes.c_int), ("rho_T", ctypes.c_double),
        ("logistic_K", ctypes.c_double),
    ]


NPHYS = 8  # (a, b, d, gamma, r, p1, p2, p3)
GROWTH = {"exp": 0, "poly4": 1, "logistic": 2}


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_chain_randoms.argtypes = [ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_uint32, dp, dp]
        L.orc_chain_randoms_from.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                             ctypes.c_uint32, dp, dp]
        L.orc_chain_randoms_pt.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                           ctypes.c_uint32, ctypes.c_uint32, dp, dp]
        L.orc_solve1d_thomas.argtypes = [ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, dp, dp]
        L.orc_dct_matrix.argtypes = [ctypes.c_int, dp]
        L.orc_laplacian_eig.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_laplacian_eig.restype = ctypes.c_double
        L.orc_solve2d_dct.argtypes = [ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, dp, dp]
        L.orc_solve2d_cg.argtypes = [ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, dp, dp, ctypes.c_double,
                                     ctypes.c_int]
        L.orc_solve2d_cg.restype = ctypes.c_int
        L.orc_solve2d_cg_var.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp,
                                         ctypes.c_double, ctypes.c_int]
        L.orc_solve2d_cg_var.restype = ctypes.c_int
        L.orc_growth.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_forward.argtypes = [ctypes.POINTER(_Problem), dp, dp, dp, dp, dp]
        L.orc_forward.restype = ctypes.c_uint32
        L.orc_forward_batch.argtypes = [ctypes.POINTER(_Problem), ctypes.c_int,
                                        dp, dp, u32p, dp, ctypes.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


# --------------------------------------------------------------------------
# Random numbers (Philox4x32-10, Salmon et al. 2011)
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """One Philox4x32-10 block.  Pinned by the published known-answer values."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_u32p(c), _u32p(k), _u32p(out))
    return out


def chain_randoms(seed: int, n_chains: int, step: int, first: int = 0, point: int = 0):
    """Normals [C][6] and uniforms [C][2] of every chain at one MCMC step
    (counters (first + chain, step, 0|1, point), key = seed; first is the
    global index of chain 0 when chains are split over processes, point the
    index of a point of the multi-proposal step, 0 otherwise).  Pinned by
    moment and distribution tests and by the Philox known-answer values."""
    normals = np.zeros((n_chains, 6))
    uniforms = np.zeros((n_chains, 2))
    lib().orc_chain_randoms_pt(ctypes.c_uint64(seed), first, n_chains, step, point,
                               _dp(normals), _dp(uniforms))
    return normals, uniforms


# --------------------------------------------------------------------------
# Implicit solves (Sec. 3.1.1)
# --------------------------------------------------------------------------
def solve1d_thomas(alpha, beta_h, rhs):
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    x = np.zeros_like(rhs)
    lib().orc_solve1d_thomas(rhs.size, alpha, beta_h, _dp(rhs), _dp(x))
    return x


def dct_matrix(n):
    c = np.zeros((n, n))
    lib().orc_dct_matrix(n, _dp(c))
    return c


def laplacian_eig(n, k):
    return lib().orc_laplacian_eig(n, k)


def solve2d_dct(alpha, beta_h, rhs):
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    x = np.zeros_like(rhs)
    lib().orc_solve2d_dct(rhs.shape[0], alpha, beta_h, _dp(rhs), _dp(x))
    return x


def solve2d_cg(alpha, beta_h, rhs, rtol=1e-14, max_iter=None):
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    x = np.zeros_like(rhs)
    n = rhs.shape[0]
    it = lib().orc_solve2d_cg(n, alpha, beta_h, _dp(rhs), _dp(x), rtol,
                              max_iter or 50 * n * n)
    return x, it


def solve2d_cg_var(alpha, beta_h, rhs, rtol=1e-14, max_iter=None):
    """[diag(alpha) - beta_h Lap_h] x = rhs in 2-D by plain CG (the operator
    of the paper's semi-implicit step, Sec. 3.1.1).  Pinned against a dense
    solve."""
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    al = np.ascontiguousarray(np.broadcast_to(alpha, rhs.shape), dtype=np.float64)
    x = np.zeros_like(rhs)
    n = rhs.shape[0]
    it = lib().orc_solve2d_cg_var(n, _dp(al), beta_h, _dp(rhs), _dp(x), rtol,
                                  max_iter or 50 * n * n)
    return x, it


# --------------------------------------------------------------------------
# Forward model + log-likelihood (eq. (schnakenberg), (reactions), (logl))
# --------------------------------------------------------------------------
class Problem:
    """A forward problem: grid, time stepping, initial state, observations.

    ``obs_steps`` are step indices (1..n_steps) at which the observed fields
    (``field_mask`` bit 0 = u, bit 1 = v) are compared with ``y`` of shape
    [n_obs][n observed fields][N] (1-D) or [n_obs][fields][N][N] (2-D).
    """

    def __init__(self, dim, n, tau, n_steps, u0, v0, y=None, obs_steps=None,
                 field_mask=1, sigma=1.0, m_growth=None, w_max=100.0,
                 solver="dct", scheme="imex", growth="exp", rho_T=1.0, logistic_K=1.0):
        self.dim, self.n, self.tau, self.n_steps = dim, n, tau, n_steps
        shape = (n,) if dim == 1 else (n, n)
        self.u0 = np.ascontiguousarray(np.broadcast_to(u0, shape), np.float64)
        self.v0 = np.ascontiguousarray(np.broadcast_to(v0, shape), np.float64)
        self.obs_steps = np.ascontiguousarray(
            obs_steps if obs_steps is not None else [], dtype=np.int32)
        nf = bin(field_mask & 3).count("1")
        if y is None:
            y = np.zeros((len(self.obs_steps), nf) + shape)
        self.y = np.ascontiguousarray(y, dtype=np.float64)
        assert self.y.size == len(self.obs_steps) * nf * int(np.prod(shape))
        self.field_mask, self.sigma = field_mask, sigma
        self.m_growth = dim if m_growth is None else m_growth
        self.w_max = w_max
        self.solver = {"dct": 0, "cg": 1}[solver]
        # "imex" (reaction explicit) or "picard" (the paper's semi-implicit step)
        self.scheme = {"imex": 0, "picard": 1}[scheme]
        # law of rho(t): "exp" (r = theta[4]), "poly4" (Example 1's polynomial,
        # theta[5:8] and rho_T) or "logistic" (rate theta[4], capacity logistic_K)
        self.growth = GROWTH[growth]
        self._c = _Problem(
            dim, n, n_steps, tau, self.m_growth, len(self.obs_steps),
            self.obs_steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            field_mask, _dp(self.y), sigma, _dp(self.u0), _dp(self.v0),
            w_max, self.solver, self.scheme, self.growth, rho_T, logistic_K)

    @property
    def shape(self):
        return (self.n,) if self.dim == 1 else (self.n, self.n)

    def forward(self, theta, want_obs=False):
        """Solve at theta = (a, b, d, gamma, r[, p1, p2, p3]); returns (phi,
        status, u, v) and, with want_obs, also the observed fields at the
        observation steps ([n_obs][observed fields][...])."""
        th = np.zeros(NPHYS)
        th[: len(theta)] = theta
        u = np.zeros(self.shape)
        v = np.zeros(self.shape)
        obs = np.zeros(self.y.shape) if want_obs else None
        phi = ctypes.c_double(0.0)
        st = lib().orc_forward(ctypes.byref(self._c), _dp(th),
                               ctypes.byref(phi), _dp(u), _dp(v),
                               _dp(obs) if want_obs else ctypes.POINTER(ctypes.c_double)())
        if want_obs:
            return phi.value, int(st), u, v, obs
        return phi.value, int(st), u, v

    def forward_batch(self, thetas, n_threads=None, want_fields=False):
        """Solves for thetas [B][5 or 8] on host threads; returns (phi, status[, fields])."""
        th = np.ascontiguousarray(thetas, dtype=np.float64)
        if th.shape[1] < NPHYS:
            th = np.concatenate([th, np.zeros((th.shape[0], NPHYS - th.shape[1]))], 1)
        B = th.shape[0]
        phi = np.zeros(B)
        status = np.zeros(B, dtype=np.uint32)
        fields = np.zeros((B, 2) + self.shape) if want_fields else None
        nt = n_threads or os.cpu_count() or 1
        lib().orc_forward_batch(
            ctypes.byref(self._c), B, _dp(th), _dp(phi), _u32p(status),
            _dp(fields) if want_fields else ctypes.POINTER(ctypes.c_double)(),
            nt)
        if want_fields:
            return phi, status, fields
        return phi, status


def growth(kind, theta, t, T, rho_T=1.0, logistic_K=1.0):
    """(rho(t), rho'(t) / rho(t)) of the growth law `kind` (see Problem)."""
    th = np.zeros(NPHYS)
    th[: len(theta)] = theta
    rho, q = ctypes.c_double(0.0), ctypes.c_double(0.0)
    lib().orc_growth(GROWTH[kind], _dp(th), rho_T, logistic_K, T, t, ctypes.byref(rho),
                     ctypes.byref(q))
    return rho.value, q.value


def poly4_positive(p, rho_T, n_check=1000):
    """Whether Example 1's polynomial rho(s) = 1 + p1 s + p2 s^2 + p3 s^3 +
    p4 s^4 (p4 = rho_T - 1 - p1 - p2 - p3) is positive at s = k / n_check,
    k = 0..n_check: the support of the growth prior (rho > 0 on [0, T]).
    p: [..., 3]."""
    p = np.asarray(p, dtype=np.float64)
    p1, p2, p3 = p[..., 0:1], p[..., 1:2], p[..., 2:3]
    p4 = rho_T - 1.0 - p1 - p2 - p3
    sv = np.arange(n_check + 1) / n_check
    rho = 1.0 + sv * (p1 + sv * (p2 + sv * (p3 + sv * p4)))
    return np.all(rho > 0.0, axis=-1)


def steady_state(a, b):
    """Homogeneous steady state (u*, v*) = (a + b, b / (a + b)^2) of the
    kinetics of eq. (reactions) (Sec. 3.1.1 and 3.1.2)."""
    return a + b, b / (a + b) ** 2
