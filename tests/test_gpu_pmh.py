"""The multi-proposal parallel Metropolis-Hastings step (Sec. 2.1,
Algorithm 2) through the C ABI against the oracle's: the 1-D FP64 workload
(deterministic solves), 4 chains with 4 proposals per step, the same random
streams on both sides -> the same draws from the (N+1)-point stationary
distribution and the same samples; the counters and the argument checks."""
import numpy as np
import pytest

import oracle
from oracle import mcmc
import paper_1605_04718_gb300 as rd
import rd_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def test_parallel_proposals_match_oracle():
    from tests.test_gpu_parity import _problem_1d
    p, P = _problem_1d(2000)
    C, N, S = 4, 4, 25
    theta0 = rd_synth.chain_starts([0.1, 0.9], C, seed=31)
    c = rd.rd_chains_create(p, theta0, 555, [0.02, 0.02], capacity=N * S)
    rd.rd_chains_set_parallel_proposals(c, N)
    rd.rd_chains_run(c, S)
    s_gpu, counters = rd.rd_chains_read_samples(c, N * S, 2, C)
    m = mcmc.Model([0, 1], np.array([0.1, 0.9, 10.0, 200.0, 0.0]), ["uniform"] * 2,
                   np.array([0.0, 0.0]), np.array([1.0, 2.0]), ["linear"] * 2,
                   np.array([0.02, 0.02]))
    ch = mcmc.ParallelChains(m, theta0, 555, lambda th: P.forward_batch(th), n_prop=N)
    s_orc = ch.run(S)
    assert s_gpu.shape == s_orc.shape == (N * S, 2, C)
    assert np.allclose(s_gpu, s_orc, rtol=1e-9, atol=1e-12)
    assert counters[0] == C * N * S and counters[2] == ch.n_acc
    assert counters[3] == ch.n_solves
    # the sample buffer counts samples: N per step
    with pytest.raises(rd.RdError):
        rd.rd_chains_run(c, S + 1)
    with pytest.raises(rd.RdError):
        rd.rd_chains_set_parallel_proposals(c, rd.RD_PMH_MAX_PROPOSALS + 1)
    s = rd.rd_surrogate_create(p, 1)
    with pytest.raises(rd.RdError):
        rd.rd_chains_set_surrogate(c, s)
    rd.rd_chains_set_parallel_proposals(c, 0)  # back to Algorithm 1
    rd.rd_chains_run(c, 1)
    rd.rd_surrogate_destroy(s)
    rd.rd_chains_destroy(c)
    rd.rd_problem_destroy(p)


def test_turing_prior_chains_match_oracle():
    """The Turing-space prior (Sec. 3.1.2 Case 2) with wide steps, so that
    proposals leave the space, under Algorithms 1 and 2: the same samples as
    the oracle's chains with the same prior."""
    from tests.test_gpu_parity import _problem_1d
    p, P = _problem_1d(1000)
    rd.rd_set_turing_prior(p, True)
    C, S, step = 4, 20, [0.25, 0.25]
    theta0 = rd_synth.chain_starts([0.1, 0.9], C, seed=41)
    m = mcmc.Model([0, 1], np.array([0.1, 0.9, 10.0, 200.0, 0.0]), ["uniform"] * 2,
                   np.array([0.0, 0.0]), np.array([1.0, 2.0]), ["linear"] * 2,
                   np.array(step), turing=True)
    for N in (0, 3):
        c = rd.rd_chains_create(p, theta0, 99, step, capacity=max(N, 1) * S)
        if N:
            rd.rd_chains_set_parallel_proposals(c, N)
            ch = mcmc.ParallelChains(m, theta0, 99, lambda th: P.forward_batch(th), n_prop=N)
        else:
            ch = mcmc.Chains(m, theta0, 99, lambda th: P.forward_batch(th))
        rd.rd_chains_run(c, S)
        s_gpu, counters = rd.rd_chains_read_samples(c, max(N, 1) * S, 2, C)
        s_orc = ch.run(S)
        assert np.allclose(s_gpu, s_orc, rtol=1e-9, atol=1e-12)
        assert counters[3] == ch.n_solves < counters[0]  # some proposals left the space
        assert np.all(mcmc.in_turing_space(s_gpu[:, 0], s_gpu[:, 1], 10.0))
        rd.rd_chains_destroy(c)
    rd.rd_problem_destroy(p)
