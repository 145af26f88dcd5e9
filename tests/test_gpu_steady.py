"""The steady-state forward map (the measurement protocol of Sec. 3.1.2) on
the GPU, through the C ABI, against the oracle's protocol: the step T at
which the discrete time derivative's L2 norm falls below the threshold, the
stationary fields, the 2T confirmation, and Phi against data taken at the
steady state; in 1-D (FP64 Thomas) and 2-D (FP32 eigenbasis on CUDA cores)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1605_04718_gb300 as rd
import rd_synth
from oracle import protocol
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
A, B_ = 0.126779, 0.792366  # Table 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def _gpu(dim, n, tau, cap, u0, v0, y, sigma, theta, threshold, confirm=True):
    prec = rd.RD_PREC_F64 if dim == 1 else rd.RD_PREC_F32
    desc = rd.make_desc(dim, [n], tau, cap, [0, 1], [A, B_, 10.0, 200.0, 0.0],
                        [rd.RD_PRIOR_UNIFORM] * 2, [0.0, 0.0], [1.0, 2.0],
                        [rd.RD_STEP_LINEAR] * 2, precision=prec)
    p = rd.rd_problem_create(desc)
    rd.rd_set_initial_state(p, 0, u0, v0)
    rd.rd_set_observations(p, 0, [cap], 3, y, sigma)
    rd.rd_set_steady_state(p, threshold, confirm)
    Bn = theta.shape[0]
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    phi = torch.zeros(Bn, dtype=torch.float64, device=DEV)
    st = torch.zeros(Bn, dtype=torch.int32, device=DEV)
    steps = torch.zeros(Bn, dtype=torch.int32, device=DEV)
    shape = (Bn, 2, n) if dim == 1 else (Bn, 2, n, n)
    fl = torch.zeros(shape, dtype=torch.float64 if dim == 1 else torch.float32, device=DEV)
    rd.rd_evaluate_batch_steady(p, th, phi, st, steps, fields=fl)
    rd.rd_sync(p)
    out = (phi.cpu().numpy(), st.cpu().numpy(), steps.cpu().numpy(), fl.double().cpu().numpy())
    return p, out


def _oracle(dim, n, tau, theta, u0, v0, threshold):
    return protocol.evolve_to_steady_state(dim, n, tau, list(theta) + [10.0, 200.0], u0, v0,
                                           threshold=threshold)


def _data(dim, n, tau, threshold, seed):
    if dim == 1:
        u0, v0 = protocol.paper_initial_state(dim, n, A, B_)
    else:
        # eq. (ic_numerical) is symmetric under (x, y) -> (1 - x, 1 - y) and its
        # symmetric pattern drifts slowly once rounding breaks the symmetry
        # (FP32 breaks it sooner than FP64); seeded noise on the homogeneous
        # steady state gives a generic pattern, stored in FP32 as the GPU does
        us, vs = oracle.steady_state(A, B_)
        noise = rd_synth.uniform_noise((2, n, n), seed, 0.01)
        u0 = (us + noise[0]).astype(np.float32).astype(np.float64)
        v0 = (vs + noise[1]).astype(np.float32).astype(np.float64)
    ref = _oracle(dim, n, tau, [A, B_], u0, v0, threshold)
    rng = np.random.default_rng(seed)
    yu, sigma = protocol.range_noise(ref["u"], 0.05, rng)
    yv = ref["v"] + rng.normal(0.0, sigma, ref["v"].shape)
    y = np.stack([yu, yv])
    if dim == 2:
        y = y.astype(np.float32).astype(np.float64)
    return u0, v0, y, sigma, ref


def test_steady_state_1d_matches_the_oracle_protocol():
    n, tau, thr = 32, 1e-4, 1e-5
    u0, v0, y, sigma, _ = _data(1, n, tau, thr, seed=3)
    theta = np.array([[A, B_], [A * 1.02, B_], [A, B_ * 0.99]])
    p, (phi, st, steps, fl) = _gpu(1, n, tau, 400000, u0, v0, y, sigma, theta, thr)
    for i, th in enumerate(theta):
        ref = _oracle(1, n, tau, th, u0, v0, thr)
        assert ref["stationary"]
        assert st[i] == 0
        assert abs(int(steps[i]) - ref["steps_T"]) <= 1, (steps[i], ref["steps_T"])
        assert H.rel_l2(fl[i, 0], ref["u"]) < 1e-8 and H.rel_l2(fl[i, 1], ref["v"]) < 1e-8
        phi_o = ((y[0] - ref["u"]) ** 2 + (y[1] - ref["v"]) ** 2).sum() / (2 * sigma**2)
        assert abs(phi[i] - phi_o) <= 1e-6 * phi_o
    # a cap below T: no steady state reached
    p2, (phi2, st2, steps2, _) = _gpu(1, n, tau, 1000, u0, v0, y, sigma, theta[:1], thr)
    assert st2[0] & rd.RD_P_NOT_CONVERGED and np.isinf(phi2[0]) and steps2[0] == 0
    for h in (p, p2):
        rd.rd_problem_destroy(h)


def test_steady_state_2d_matches_the_oracle_protocol():
    """FP32 fields: rounding keeps forcing the pattern's slowest modes, so the
    time-derivative norm of an FP32 solve levels off well above the FP64 one
    near the steady state (a 1e-3 threshold was reached 60 % later than in
    FP64); the threshold here is 1e-2, where the norm still decays fast, and
    T may differ by 10 % (the paper's 1e-5 needs the FP64 path, 1-D)."""
    n, tau, thr = 32, 2.5e-4, 1e-2
    u0, v0, y, sigma, ref = _data(2, n, tau, thr, seed=4)
    assert ref["stationary"]
    theta = np.array([[A, B_]])
    p, (phi, st, steps, fl) = _gpu(2, n, tau, 300000, u0, v0, y.reshape(2, n, n), sigma,
                                   theta, thr)
    assert st[0] == 0
    T = int(steps[0])
    assert abs(T - ref["steps_T"]) <= 0.1 * ref["steps_T"], (T, ref["steps_T"])
    # the state the GPU stopped in against the oracle's state at the same step
    # (the approach to the steady state is slow, so states a few hundred steps
    # apart differ by more than the FP32 tolerance)
    P = oracle.Problem(2, n, tau, T, u0, v0, y=y.reshape(1, 2, n, n), obs_steps=[T],
                       field_mask=3, sigma=sigma)
    phi_o, _, uo, vo = P.forward([A, B_, 10.0, 200.0, 0.0])
    w_o = np.stack([uo, vo]).reshape(2, -1)
    assert H.rel_l2(fl[0].reshape(2, -1), w_o) < 1e-3
    assert abs(phi[0] - phi_o) <= H.phi_tolerance(y.reshape(-1), w_o.reshape(-1), sigma)
    with pytest.raises(rd.RdError):  # 128^2 is beyond the CUDA-core kernel's copy
        d128 = H.small_dataset(128, 4, seed=1)
        q = H.gpu_problem([d128])
        try:
            rd.rd_set_steady_state(q, 1e-5)
        finally:
            rd.rd_problem_destroy(q)
    rd.rd_problem_destroy(p)
