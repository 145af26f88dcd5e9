"""Example 1 (Sec. 3.1.1): identification of the domain growth rho(t) on the
1-D growing interval, on the GPU through the C ABI against the FP64 oracle.
The model parameters inferred are Example 1's three polynomial degrees of
freedom (p1, p2, p3) with rho(0) = 1 and rho(T) = rho_T fixed; the kinetics
are the paper's a = 0.1, b = 0.9, d = 10, gamma = 1000; the step is the
paper's semi-implicit one (FP64 Thomas per proposal); the data are the stored
exponential-law observations at T = 600 (6e6 steps)."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1605_04718_gb300 as rd
import rd_synth
from oracle import mcmc
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
KIN = [0.1, 0.9, 10.0, 1000.0, 0.0]
BOX = ([-2.0, -6.0, -6.0], [4.0, 6.0, 6.0])  # uniform prior box on (p1, p2, p3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def _problems(name, n_steps, rho_T):
    spec = rd_synth.DATASETS[name]
    d = H.load_dataset(name)
    desc = rd.make_desc(1, [spec["n"]], spec["tau"], n_steps, [5, 6, 7], KIN,
                        [rd.RD_PRIOR_UNIFORM] * 3, BOX[0], BOX[1], [rd.RD_STEP_LINEAR] * 3,
                        solver=rd.RD_SOLVER_THOMAS, growth=rd.RD_GROWTH_POLY4, rho_T=rho_T)
    p = rd.rd_problem_create(desc)
    rd.rd_set_scheme(p, rd.RD_SCHEME_PICARD)
    rd.rd_set_initial_state(p, 0, d["u0"], d["v0"])
    rd.rd_set_observations(p, 0, [n_steps], 3, d["y"], float(d["sigma"]))
    P = oracle.Problem(1, spec["n"], spec["tau"], n_steps, d["u0"], d["v0"], y=d["y"],
                       obs_steps=[n_steps], field_mask=3, sigma=float(d["sigma"]),
                       scheme="picard", growth="poly4", rho_T=rho_T)
    return p, P


def _eval(p, theta, n):
    B = theta.shape[0]
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    phi = torch.zeros(B, dtype=torch.float64, device=DEV)
    st = torch.zeros(B, dtype=torch.int32, device=DEV)
    fl = torch.zeros((B, 2, n), dtype=torch.float64, device=DEV)
    rd.rd_evaluate_batch(p, th, phi, st, fields=fl)
    rd.rd_sync(p)
    return phi.cpu().numpy(), st.cpu().numpy(), fl.cpu().numpy()


def _full(theta):
    return np.concatenate([np.tile(KIN, (len(theta), 1)), theta], 1)


def _draws(B, rho_T, seed):
    """Uniform draws from the prior box, kept where rho > 0 on [0, T]."""
    out = []
    rng = np.random.default_rng(seed)
    while len(out) < B:
        p = rng.uniform(BOX[0], BOX[1])
        if oracle.poly4_positive(p, rho_T):
            out.append(p)
    return np.array(out)


def test_fields_and_phi_match_oracle_bit_for_bit():
    """60000 steps (T = 6, the polynomial law stretched over it) for 16 prior
    draws: the GPU's explicitly rounded FP64 step reproduces the oracle's
    fields bit for bit; Phi (summed in another order) within 1e-12."""
    rho_T = 1.3
    p, P = _problems("rd1d_e1_exp", 60000, rho_T)
    theta = _draws(16, rho_T, seed=1)
    phi, st, fl = _eval(p, theta, 100)
    po, so, fo = P.forward_batch(_full(theta), want_fields=True)
    for i in range(len(theta)):
        assert st[i] == so[i] == 0
        assert np.array_equal(fl[i], fo[i]), (i, H.rel_l2(fl[i], fo[i]))
        assert abs(phi[i] - po[i]) <= 1e-12 * po[i]
    rd.rd_problem_destroy(p)


def test_long_horizon_stays_bit_identical():
    """600000 steps (T = 60) at gamma = 1000 on the growing interval, where
    the pattern's peak insertions amplify any rounding difference: the
    fields still agree bit for bit (the paper's T = 600 takes 6e6 such steps,
    about 10 minutes per proposal in FP64 on the GPU, so the test stops at a
    tenth of it)."""
    rho_T = 1.3
    p, P = _problems("rd1d_e1_exp", 600000, rho_T)
    theta = np.concatenate([[[0.3, 0.0, 0.0]], _draws(1, rho_T, seed=2)], 0)
    phi, st, fl = _eval(p, theta, 100)
    po, so, fo = P.forward_batch(_full(theta), want_fields=True)
    for i in range(len(theta)):
        assert st[i] == so[i] == 0
        assert np.array_equal(fl[i], fo[i]), (i, H.rel_l2(fl[i], fo[i]))
    rd.rd_problem_destroy(p)


def test_growth_chains_match_oracle_and_respect_the_support():
    """Random-walk chains over (p1, p2, p3) on the GPU and in the oracle with
    the same random numbers: the same samples; proposals with rho <= 0
    somewhere on [0, T] are rejected without a solve.  The horizon (2000
    steps) ends before the pattern forms: later, the last-bit differences of
    the two platforms' Box-Muller proposals grow like any perturbation and
    can flip a decision."""
    rho_T = 1.3
    p, P = _problems("rd1d_e1_exp", 2000, rho_T)
    C, S = 4, 20
    step = [0.3, 0.6, 0.6]
    theta0 = _draws(C, rho_T, seed=3)
    c = rd.rd_chains_create(p, theta0, 77, step, capacity=S)
    rd.rd_chains_run(c, S)
    s_gpu, cnt = rd.rd_chains_read_samples(c, S, 3, C)
    m = mcmc.Model([5, 6, 7], np.array(KIN), ["uniform"] * 3, np.array(BOX[0]),
                   np.array(BOX[1]), ["linear"] * 3, np.array(step), poly_rho_T=rho_T)
    ch = mcmc.Chains(m, theta0, 77, lambda th: P.forward_batch(th))
    s_orc = ch.run(S)
    # proposals from Box-Muller may differ in the last bit (each platform's
    # log / sin / cos), so samples agree to rounding, decisions exactly
    assert np.allclose(s_gpu, s_orc, rtol=1e-12, atol=1e-14)
    assert cnt[2] == ch.n_acc
    assert np.all(oracle.poly4_positive(s_gpu.transpose(0, 2, 1), rho_T))
    rd.rd_chains_destroy(c)
    with pytest.raises(rd.RdError):  # the polynomial law is 1-D only
        desc = rd.make_desc(2, [32], 1e-4, 10, [5, 6, 7], KIN, [rd.RD_PRIOR_UNIFORM] * 3,
                            BOX[0], BOX[1], [rd.RD_STEP_LINEAR] * 3,
                            growth=rd.RD_GROWTH_POLY4, rho_T=rho_T)
        rd.rd_problem_create(desc)
    rd.rd_problem_destroy(p)
