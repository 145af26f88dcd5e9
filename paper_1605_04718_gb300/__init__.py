"""Python binding of the GB300 library for Bayesian identification of
Schnakenberg reaction-diffusion parameters (arXiv:1605.04718).

Argument marshalling only: every function forwards to the ``extern "C"`` entry
point of the same name in ``include/rdbayes.h`` (built into
``_build/librdbayes.so`` by ``build.py``).  Every step of the path runs in
the library's CUDA kernels; there is no CPU fallback, and importing a function
that needs the library raises if the library has not been built.

Device arrays are torch CUDA tensors (PyTorch supplies device memory and the
stream); host arrays are numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librdbayes.so")

RD_OK, RD_EINVAL, RD_ENOMEM, RD_ECUDA, RD_ESTATE, RD_ETIMEOUT = range(6)
RD_P_OK, RD_P_OUT_OF_SUPPORT, RD_P_NONFINITE, RD_P_NOT_CONVERGED, RD_P_NOT_SOLVED = 0, 1, 2, 4, 8
RD_SOLVER_AUTO, RD_SOLVER_THOMAS, RD_SOLVER_DCT_SIMT, RD_SOLVER_DCT_TC = range(4)
RD_PRIOR_UNIFORM, RD_PRIOR_LOGNORMAL = 0, 1
RD_STEP_LINEAR, RD_STEP_LOG = 0, 1
RD_PREC_F64, RD_PREC_F32 = 0, 1
RD_SCHEME_IMEX, RD_SCHEME_PICARD = 0, 1
RD_KERNEL_DEFAULT, RD_KERNEL_SIMT, RD_KERNEL_TC_STACKED, RD_KERNEL_TC_RESIDENT, RD_KERNEL_CG = range(5)
RD_MAX_SIZES, RD_MAX_OBS, RD_NPARAM, RD_NPHYS = 4, 8, 5, 8
RD_GROWTH_NONE, RD_GROWTH_EXP, RD_GROWTH_POLY4 = 0, 1, 2
RD_NOALLOC_MAX_BATCH = 65536
RD_PMH_MAX_PROPOSALS = 16
RD_SURROGATE_WIDTH = 256
SURROGATE_IN = 16  # padded network inputs

# Every entry point declared in include/rdbayes.h.
EXPORTS = (
    "rd_problem_create", "rd_problem_destroy", "rd_set_stream",
    "rd_set_initial_state", "rd_set_observations", "rd_evaluate_batch",
    "rd_evaluate_batch_host", "rd_evaluate_batch_noalloc", "rd_chains_create", "rd_chains_destroy",
    "rd_chains_run", "rd_chains_read_samples", "rd_chains_get_state",
    "rd_chains_checkpoint", "rd_chains_restore", "rd_sync", "rd_last_error",
    "rd_surrogate_create", "rd_surrogate_destroy", "rd_surrogate_train",
    "rd_surrogate_predict", "rd_surrogate_loss_grad", "rd_surrogate_get_params",
    "rd_surrogate_set_params", "rd_chains_set_surrogate", "rd_chains_set_proposal",
    "rd_set_size_kernel", "rd_get_size_kernel", "rd_autotune", "rd_chains_set_first_chain",
    "rd_chains_set_parallel_proposals", "rd_set_turing_prior", "rd_set_scheme",
    "rd_set_wait_limit", "rd_debug_stall_at_step", "rd_set_steady_state",
    "rd_evaluate_batch_steady", "rd_set_size_schedule", "rd_get_size_schedule",
)


class RdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rdbayes error {code}: {msg}")
        self.code = code


class rd_problem_desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n_sizes", ctypes.c_int),
        ("nx", ctypes.c_int * RD_MAX_SIZES), ("tau", ctypes.c_double),
        ("n_steps", ctypes.c_int), ("precision", ctypes.c_int),
        ("solver", ctypes.c_int), ("growth", ctypes.c_int),
        ("n_params", ctypes.c_int), ("param_map", ctypes.c_int * RD_NPARAM),
        ("fixed", ctypes.c_double * RD_NPARAM),
        ("prior_kind", ctypes.c_int * RD_NPARAM),
        ("prior_p0", ctypes.c_double * RD_NPARAM),
        ("prior_p1", ctypes.c_double * RD_NPARAM),
        ("step_space", ctypes.c_int * RD_NPARAM), ("w_max", ctypes.c_double),
        ("fixed_poly", ctypes.c_double * 3), ("rho_T", ctypes.c_double),
    ]


class rd_train_desc(ctypes.Structure):
    _fields_ = [
        ("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
        ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
        ("weight_decay", ctypes.c_double), ("holdout_frac", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


_lib = None


def load():
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.rd_problem_create.argtypes = [ctypes.POINTER(rd_problem_desc), vp, ctypes.POINTER(vp)]
    L.rd_problem_destroy.argtypes = [vp]
    L.rd_set_stream.argtypes = [vp, vp]
    L.rd_set_initial_state.argtypes = [vp, i, vp, vp]
    L.rd_set_observations.argtypes = [vp, i, i, vp, i, vp, d]
    L.rd_evaluate_batch.argtypes = [vp, i, vp, vp, vp, vp, vp]
    L.rd_evaluate_batch_host.argtypes = [vp, i, vp, vp, vp, vp]
    L.rd_evaluate_batch_noalloc.argtypes = [vp, i, vp, vp, vp, vp, vp]
    L.rd_chains_create.argtypes = [vp, i, vp, ctypes.c_uint64, vp, vp, i, ctypes.POINTER(vp)]
    L.rd_chains_destroy.argtypes = [vp]
    L.rd_chains_run.argtypes = [vp, i]
    L.rd_chains_read_samples.argtypes = [vp, vp, ctypes.c_size_t,
                                         ctypes.POINTER(ctypes.c_size_t), vp]
    L.rd_chains_get_state.argtypes = [vp, vp, vp]
    L.rd_chains_checkpoint.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.rd_chains_restore.argtypes = [vp, vp, ctypes.c_size_t]
    L.rd_sync.argtypes = [vp]
    L.rd_surrogate_create.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(vp)]
    L.rd_surrogate_destroy.argtypes = [vp]
    L.rd_surrogate_train.argtypes = [vp, i, vp, vp, ctypes.POINTER(rd_train_desc), vp]
    L.rd_surrogate_predict.argtypes = [vp, i, vp, vp]
    L.rd_surrogate_loss_grad.argtypes = [vp, i, vp, vp, ctypes.POINTER(ctypes.c_double), vp]
    L.rd_surrogate_get_params.argtypes = [vp, vp, ctypes.c_size_t,
                                          ctypes.POINTER(ctypes.c_size_t), vp]
    L.rd_surrogate_set_params.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.rd_chains_set_surrogate.argtypes = [vp, vp]
    L.rd_chains_set_proposal.argtypes = [vp, vp]
    L.rd_set_wait_limit.argtypes = [vp, d]
    L.rd_set_steady_state.argtypes = [vp, d, i]
    L.rd_evaluate_batch_steady.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    L.rd_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "rd_last_error":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(code):
    if code != RD_OK:
        msg = load().rd_last_error().decode(errors="replace")
        raise RdError(code, msg)


def _host_ptr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


def make_desc(dim, nx, tau, n_steps, param_map, fixed, prior_kind, prior_p0,
              prior_p1, step_space, solver=RD_SOLVER_AUTO, growth=0,
              precision=None, w_max=100.0, rho_T=1.0):
    """Fills an rd_problem_desc (see include/rdbayes.h for each field)."""
    desc = rd_problem_desc()
    desc.dim = dim
    nx = list(nx)
    desc.n_sizes = len(nx)
    for s, n in enumerate(nx):
        desc.nx[s] = n
    desc.tau = tau
    desc.n_steps = n_steps
    desc.precision = (RD_PREC_F64 if dim == 1 else RD_PREC_F32) if precision is None else precision
    desc.solver = solver
    desc.growth = growth
    desc.n_params = len(param_map)
    for j in range(len(param_map)):
        desc.param_map[j] = param_map[j]
        desc.prior_kind[j] = prior_kind[j]
        desc.prior_p0[j] = prior_p0[j]
        desc.prior_p1[j] = prior_p1[j]
        desc.step_space[j] = step_space[j]
    for k in range(RD_NPARAM):
        desc.fixed[k] = fixed[k]
    for k in range(3):  # p1..p3 of the polynomial growth law
        desc.fixed_poly[k] = fixed[RD_NPARAM + k] if len(fixed) > RD_NPARAM + k else 0.0
    desc.w_max = w_max
    desc.rho_T = rho_T
    return desc


def rd_problem_create(desc, stream=None):
    h = ctypes.c_void_p()
    _check(load().rd_problem_create(ctypes.byref(desc), _stream_handle(stream), ctypes.byref(h)))
    return h


def rd_problem_destroy(p):
    _check(load().rd_problem_destroy(p))


def rd_set_stream(p, stream=None):
    _check(load().rd_set_stream(p, _stream_handle(stream)))


def rd_set_initial_state(p, size_idx, u0, v0):
    u0, pu = _host_ptr(u0, np.float64)
    v0, pv = _host_ptr(v0, np.float64)
    _check(load().rd_set_initial_state(p, size_idx, pu, pv))


def rd_set_observations(p, size_idx, obs_steps, field_mask, y, sigma):
    st, ps = _host_ptr(obs_steps, np.int32)
    y, py = _host_ptr(y, np.float64)
    _check(load().rd_set_observations(p, size_idx, len(st), ps, field_mask, py, sigma))


def rd_evaluate_batch(p, theta, loglik, status, size_idx=None, fields=None):
    """theta [B][P] float64, loglik [B] float64, status [B] int32 (bit
    pattern of uint32), size_idx [B] int32 or None, fields or None: CUDA tensors."""
    _check(load().rd_evaluate_batch(p, theta.shape[0], _dev_ptr(theta), _dev_ptr(size_idx),
                                    _dev_ptr(loglik), _dev_ptr(status), _dev_ptr(fields)))


def rd_evaluate_batch_noalloc(p, theta, loglik, status, size_idx=None, fields=None):
    """As rd_evaluate_batch, for callers that cannot allocate device memory
    during the call: the work lists use the library's fixed device array, so
    B is limited to RD_NOALLOC_MAX_BATCH and overlapping calls must be
    serialised by the caller (see include/rdbayes.h)."""
    _check(load().rd_evaluate_batch_noalloc(p, theta.shape[0], _dev_ptr(theta), _dev_ptr(size_idx),
                                            _dev_ptr(loglik), _dev_ptr(status), _dev_ptr(fields)))


def rd_set_steady_state(p, threshold, confirm=False):
    """Steady-state forward map: solve until the time derivative's L2 norm is
    below threshold (0 = off), optionally confirmed at 2T."""
    _check(load().rd_set_steady_state(p, float(threshold), 1 if confirm else 0))


def rd_evaluate_batch_steady(p, theta, loglik, status, steps, size_idx=None, fields=None):
    """rd_evaluate_batch in steady-state mode; steps: int32 CUDA tensor [B]
    receives the step T at which each solve became stationary."""
    _check(load().rd_evaluate_batch_steady(p, theta.shape[0], _dev_ptr(theta),
                                           _dev_ptr(size_idx), _dev_ptr(loglik),
                                           _dev_ptr(status), _dev_ptr(fields), _dev_ptr(steps)))


def rd_set_scheme(p, scheme):
    _check(load().rd_set_scheme(p, scheme))


def rd_set_wait_limit(p, seconds):
    """Limit of the tensor-core solve kernels' bounded waits (default 4 s)."""
    _check(load().rd_set_wait_limit(p, float(seconds)))


def rd_debug_stall_at_step(p, step):
    """Failure-path test aid: tensor-core issuers stall at IMEX step `step`
    (-1 = off), so the launch ends with RD_ETIMEOUT after the wait limit."""
    _check(load().rd_debug_stall_at_step(p, int(step)))


def rd_set_turing_prior(p, enable=True):
    _check(load().rd_set_turing_prior(p, 1 if enable else 0))


def rd_set_size_kernel(p, size_idx, kernel):
    _check(load().rd_set_size_kernel(p, size_idx, kernel))


def rd_set_size_schedule(p, size_idx, ctas_per_sm):
    """Persistent CTAs per SM of that size's launch (0 = as many as fit)."""
    _check(load().rd_set_size_schedule(p, size_idx, ctas_per_sm))


def rd_get_size_schedule(p, size_idx):
    k = ctypes.c_int(0)
    _check(load().rd_get_size_schedule(p, size_idx, ctypes.byref(k)))
    return k.value


def rd_get_size_kernel(p, size_idx):
    k = ctypes.c_int(0)
    _check(load().rd_get_size_kernel(p, size_idx, ctypes.byref(k)))
    return k.value


def rd_autotune(p, theta, n_trials=3, probe_steps=0, n_sizes=None):
    """theta: host [B][P].  Returns [n_sizes][4] seconds per proposal (SIMT,
    TC_STACKED, TC_RESIDENT, CG; NaN where not applicable)."""
    th, pt = _host_ptr(theta, np.float64)
    ns = n_sizes if n_sizes is not None else RD_MAX_SIZES
    out = np.full((RD_MAX_SIZES, 4), np.nan)
    _check(load().rd_autotune(p, th.shape[0], pt, n_trials, probe_steps,
                              out.ctypes.data_as(ctypes.c_void_p)))
    return out[:ns]


def rd_evaluate_batch_host(p, theta, size_idx=None):
    th, pt = _host_ptr(theta, np.float64)
    B = th.shape[0]
    if size_idx is not None:
        sz, psz = _host_ptr(size_idx, np.int32)
    else:
        psz = None
    phi = np.zeros(B)
    st = np.zeros(B, dtype=np.uint32)
    _check(load().rd_evaluate_batch_host(p, B, pt, psz, phi.ctypes.data_as(ctypes.c_void_p),
                                         st.ctypes.data_as(ctypes.c_void_p)))
    return phi, st


def rd_chains_create(p, theta0, seed, step, size_idx=None, capacity=1024):
    th, pt = _host_ptr(theta0, np.float64)
    sp, ps = _host_ptr(step, np.float64)
    if size_idx is not None:
        sz, psz = _host_ptr(size_idx, np.int32)
    else:
        psz = None
    h = ctypes.c_void_p()
    _check(load().rd_chains_create(p, th.shape[0], pt, ctypes.c_uint64(seed), ps, psz,
                                   capacity, ctypes.byref(h)))
    return h


def rd_chains_destroy(c):
    _check(load().rd_chains_destroy(c))


def rd_chains_run(c, n_steps):
    _check(load().rd_chains_run(c, n_steps))


def rd_chains_read_samples(c, cap_steps, n_params, n_chains):
    """Returns (samples [n][P][C], counters [4]: proposals, stage-1 survivors,
    accepted, exact solves)."""
    out = np.zeros((cap_steps, n_params, n_chains))
    n = ctypes.c_size_t(0)
    counters = np.zeros(4)
    _check(load().rd_chains_read_samples(c, out.ctypes.data_as(ctypes.c_void_p), cap_steps,
                                         ctypes.byref(n), counters.ctypes.data_as(ctypes.c_void_p)))
    return out[: n.value], counters


def rd_chains_get_state(c, n_params, n_chains):
    th = np.zeros((n_chains, n_params))
    phi = np.zeros(n_chains)
    _check(load().rd_chains_get_state(c, th.ctypes.data_as(ctypes.c_void_p),
                                      phi.ctypes.data_as(ctypes.c_void_p)))
    return th, phi


def rd_chains_checkpoint(c):
    n = ctypes.c_size_t(0)
    _check(load().rd_chains_checkpoint(c, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(load().rd_chains_checkpoint(c, buf, n.value, ctypes.byref(n)))
    return buf.raw


def rd_chains_restore(c, blob):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().rd_chains_restore(c, buf, len(blob)))


def rd_sync(p):
    _check(load().rd_sync(p))


def rd_last_error():
    return load().rd_last_error().decode(errors="replace")


# ----------------------------------------------------------------- surrogate
def rd_surrogate_create(p, seed=0):
    h = ctypes.c_void_p()
    _check(load().rd_surrogate_create(p, ctypes.c_uint64(seed), ctypes.byref(h)))
    return h


def rd_surrogate_destroy(s):
    _check(load().rd_surrogate_destroy(s))


def rd_surrogate_train(s, theta, phi, epochs=30, batch=1024, lr=1e-3, beta1=0.9, beta2=0.999,
                       weight_decay=0.0, holdout_frac=0.1, seed=0):
    """theta [n][P] float64, phi [n] float64: CUDA tensors.  Returns the report
    (train MSE, hold-out MSE, hold-out mean relative Phi error, seconds)."""
    td = rd_train_desc(epochs, batch, lr, beta1, beta2, weight_decay, holdout_frac, seed)
    rep = np.zeros(4)
    _check(load().rd_surrogate_train(s, theta.shape[0], _dev_ptr(theta), _dev_ptr(phi),
                                     ctypes.byref(td), rep.ctypes.data_as(ctypes.c_void_p)))
    return rep


def rd_surrogate_predict(s, theta, phi_tilde):
    _check(load().rd_surrogate_predict(s, theta.shape[0], _dev_ptr(theta), _dev_ptr(phi_tilde)))


def rd_surrogate_loss_grad(s, theta, target, grads=None):
    """target: float32 CUDA tensor [B]; grads: float32 CUDA tensor or None."""
    loss = ctypes.c_double(0.0)
    _check(load().rd_surrogate_loss_grad(s, theta.shape[0], _dev_ptr(theta), _dev_ptr(target),
                                         ctypes.byref(loss), _dev_ptr(grads)))
    return loss.value


def rd_surrogate_get_params(s):
    n = ctypes.c_size_t(0)
    _check(load().rd_surrogate_get_params(s, None, 0, ctypes.byref(n), None))
    buf = np.zeros(n.value, dtype=np.float32)
    norm = np.zeros(2 * RD_NPARAM + 3)
    _check(load().rd_surrogate_get_params(s, buf.ctypes.data_as(ctypes.c_void_p), n.value,
                                          ctypes.byref(n), norm.ctypes.data_as(ctypes.c_void_p)))
    return buf, norm


def rd_surrogate_set_params(s, params=None, norm=None):
    pp, pn = None, None
    if params is not None:
        params, pp = _host_ptr(params, np.float32)
    if norm is not None:
        norm, pn = _host_ptr(norm, np.float64)
    _check(load().rd_surrogate_set_params(s, pp, 0 if params is None else params.size, pn))


def rd_chains_set_surrogate(c, s):
    _check(load().rd_chains_set_surrogate(c, s))


def rd_chains_set_first_chain(c, first):
    """Global index of chain 0 in the random-number counters (sharded runs)."""
    _check(load().rd_chains_set_first_chain(c, ctypes.c_uint32(first)))


def rd_chains_set_parallel_proposals(c, n_prop):
    """Algorithm 2 with n_prop proposals per chain and step (0 = Algorithm 1);
    each step then yields n_prop samples per chain."""
    _check(load().rd_chains_set_parallel_proposals(c, n_prop))


def rd_chains_set_proposal(c, L):
    """L: [P][P] lower-triangular factor of the random-walk covariance (step space)."""
    L, pl = _host_ptr(L, np.float64)
    _check(load().rd_chains_set_proposal(c, pl))
