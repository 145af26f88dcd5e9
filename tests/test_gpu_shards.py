"""Chains split into contiguous ranges, as one process per GPU would run
them (rd_chains_set_first_chain with the range's start, the same seed): two
chain objects of 3 chains each, run one after the other on this GPU, give
bit for bit the samples of one object of 6 chains (1-D FP64 workload, whose
solves are deterministic), and chain 3 alone started at first = 3 matches the
oracle's chain 3 of a 6-chain run."""
import numpy as np
import pytest

import oracle
from oracle import mcmc
import paper_1605_04718_gb300 as rd
import rd_synth
from paper_1605_04718_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def _problem_1d(n_steps=2000):
    from tests.test_gpu_parity import _problem_1d as make
    return make(n_steps)


def _run(p, theta0, first, S, seed=77):
    c = rd.rd_chains_create(p, theta0, seed, [0.01, 0.01], capacity=S)
    if first:
        rd.rd_chains_set_first_chain(c, first)
    rd.rd_chains_run(c, S)
    s, _ = rd.rd_chains_read_samples(c, S, 2, theta0.shape[0])
    rd.rd_chains_destroy(c)
    return s


def test_two_shards_equal_one_run():
    p, P = _problem_1d()
    C, S = 6, 60
    theta0 = rd_synth.chain_starts([0.1, 0.9], C, seed=5)
    whole = _run(p, theta0, 0, S)
    parts = []
    for rank in range(2):
        first, count = shard.shard(C, 2, rank)
        parts.append(_run(p, theta0[first:first + count], first, S))
    assert np.array_equal(np.concatenate(parts, axis=-1), whole)
    with pytest.raises(rd.RdError):
        c = rd.rd_chains_create(p, theta0, 77, [0.01, 0.01], capacity=4)
        try:
            rd.rd_chains_set_first_chain(c, 2**32 - 3)  # first + C beyond 2^32
        finally:
            rd.rd_chains_destroy(c)
    # one shard against the oracle's chains at the same global indices
    m = mcmc.Model([0, 1], np.array([0.1, 0.9, 10.0, 200.0, 0.0]), ["uniform"] * 2,
                   np.array([0.0, 0.0]), np.array([1.0, 2.0]), ["linear"] * 2,
                   np.array([0.01, 0.01]))
    ch = mcmc.Chains(m, theta0[3:], 77, lambda th: P.forward_batch(th), first_chain=3)
    assert np.allclose(parts[1], ch.run(S), rtol=1e-9, atol=1e-12)
    rd.rd_problem_destroy(p)
