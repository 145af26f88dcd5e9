"""The paper's semi-implicit time step (Sec. 3.1.1, Example 1) on the GPU,
through the C ABI, against the FP64 oracle: 1-D fields and Phi on a fixed and
on a growing domain, chains with the same random streams, and the argument
checks."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mcmc
import paper_1605_04718_gb300 as rd
import rd_synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def _problem(n_steps, growth=False):
    spec = rd_synth.DATASETS["rd1d_n64"]
    ds = H.load_dataset("rd1d_n64")
    pm = [0, 1, 4] if growth else [0, 1]
    desc = rd.make_desc(1, [64], spec["tau"], n_steps, pm, [0.1, 0.9, 10.0, 200.0, 0.0],
                        [rd.RD_PRIOR_UNIFORM] * len(pm), [0.0] * len(pm),
                        [1.0, 2.0, 0.1][: len(pm)], [rd.RD_STEP_LINEAR] * len(pm),
                        solver=rd.RD_SOLVER_THOMAS, growth=1 if growth else 0)
    p = rd.rd_problem_create(desc)
    rd.rd_set_scheme(p, rd.RD_SCHEME_PICARD)
    rd.rd_set_initial_state(p, 0, ds["u0"], ds["v0"])
    rd.rd_set_observations(p, 0, [n_steps], 1, ds["y"], spec["sigma"])
    P = oracle.Problem(1, 64, spec["tau"], n_steps, ds["u0"], ds["v0"], y=ds["y"],
                       obs_steps=[n_steps], field_mask=1, sigma=spec["sigma"], scheme="picard")
    return p, P


@pytest.mark.parametrize("growth", [False, True])
def test_picard_fields_and_phi_match_oracle(growth):
    p, P = _problem(3000, growth)
    B = 8
    theta = np.column_stack([rd_synth.uniform_draws([0.05, 0.8], [0.15, 1.0], B, 7)] +
                            ([np.linspace(0.0, 0.05, B)] if growth else []))
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    phi = torch.zeros(B, dtype=torch.float64, device=DEV)
    st = torch.zeros(B, dtype=torch.int32, device=DEV)
    fl = torch.zeros((B, 2, 64), dtype=torch.float64, device=DEV)
    rd.rd_evaluate_batch(p, th, phi, st, fields=fl)
    rd.rd_sync(p)
    full = np.zeros((B, 5))
    full[:, :2] = theta[:, :2]
    full[:, 2:4] = [10.0, 200.0]
    if growth:
        full[:, 4] = theta[:, 2]
    for i in range(B):
        po, so, uo, vo = P.forward(full[i])
        assert int(st[i]) == so == 0
        assert H.rel_l2(fl[i, 0].cpu().numpy(), uo) < 1e-10
        assert H.rel_l2(fl[i, 1].cpu().numpy(), vo) < 1e-10
        assert abs(phi[i].item() - po) <= 1e-6 * abs(po)
    rd.rd_problem_destroy(p)


def test_picard_chains_match_oracle_and_argument_checks():
    p, P = _problem(1500)
    C, S = 4, 25
    theta0 = rd_synth.chain_starts([0.1, 0.9], C, seed=51)
    c = rd.rd_chains_create(p, theta0, 808, [0.01, 0.01], capacity=S)
    rd.rd_chains_run(c, S)
    s_gpu, counters = rd.rd_chains_read_samples(c, S, 2, C)
    m = mcmc.Model([0, 1], np.array([0.1, 0.9, 10.0, 200.0, 0.0]), ["uniform"] * 2,
                   np.array([0.0, 0.0]), np.array([1.0, 2.0]), ["linear"] * 2,
                   np.array([0.01, 0.01]))
    ch = mcmc.Chains(m, theta0, 808, lambda th: P.forward_batch(th))
    assert np.allclose(s_gpu, ch.run(S), rtol=1e-9, atol=1e-12)
    assert counters[2] == ch.n_acc
    rd.rd_chains_destroy(c)
    with pytest.raises(rd.RdError):
        rd.rd_set_scheme(p, 7)
    rd.rd_problem_destroy(p)
    ds2 = H.small_dataset(32, 4, seed=3)
    p2 = H.gpu_problem([ds2])
    with pytest.raises(rd.RdError):
        rd.rd_set_scheme(p2, rd.RD_SCHEME_PICARD)  # 2-D: not built
    rd.rd_problem_destroy(p2)
