"""The multi-process path on the host (no GPU): chains split over 2 and 3
gloo ranks with contiguous ranges and the global chain index in the random
counters give exactly the samples of one process running all chains, gathered
in chain order on every rank; the whole-job rate is all units over the
slowest rank's time.  Uses the oracle sampler on a linear-Gaussian toy target
as the per-rank work."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import mcmc
from paper_1605_04718_gb300 import shard

A_TOY = np.array([[1.0, 0.5], [0.2, 1.5], [0.7, -0.4]])
Y_TOY = np.array([1.0, 2.0, 0.3])
SEED, STEPS = 17, 40


def _model():
    return mcmc.Model(param_map=[0, 1], fixed=np.zeros(5), prior_kind=["uniform"] * 2,
                      prior_p0=np.array([-10.0, -10.0]), prior_p1=np.array([10.0, 10.0]),
                      step_space=["linear"] * 2, step=np.array([0.3, 0.3]))


def _phi(theta_full):
    r = Y_TOY[None, :] - theta_full[:, :2] @ A_TOY.T
    return (r * r).sum(1) / (2 * 0.5**2), np.zeros(theta_full.shape[0], np.uint32)


def _starts(n):
    return np.stack([np.linspace(-1, 1, n), np.linspace(0.5, 1.5, n)], 1)


def _rank_main(rank, world, port, n_total, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = shard.shard(n_total, world, rank)
        ch = mcmc.Chains(_model(), _starts(n_total)[first:first + count], SEED, _phi,
                         first_chain=first)
        local = ch.run(STEPS)                       # [steps][P][count]
        pooled = shard.gather_chains(local, dist)   # every rank gets all chains
        units, secs, rate = shard.aggregate_rate(count * STEPS, 1.0 + rank, dist)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), pooled=pooled,
                 agg=np.array([units, secs, rate]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges():
    for n, world in [(10, 3), (7, 2), (4096, 8), (3, 4)]:
        ranges = [shard.shard(n, world, r) for r in range(world)]
        assert sum(c for _, c in ranges) == n
        assert ranges[0][0] == 0
        for (f0, c0), (f1, _) in zip(ranges, ranges[1:]):
            assert f1 == f0 + c0
        assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        shard.shard(4, 2, 2)


def test_single_process_passthrough():
    x = np.arange(24.0).reshape(2, 3, 4)
    assert shard.gather_chains(x) is not None and np.array_equal(shard.gather_chains(x), x)
    assert shard.aggregate_rate(10.0, 2.0) == (10.0, 2.0, 5.0)


@pytest.mark.parametrize("world,n_total", [(2, 6), (3, 7)])
def test_ranks_reproduce_one_process(world, n_total):
    with tempfile.TemporaryDirectory() as out:
        mp.start_processes(_rank_main, args=(world, _free_port(), n_total, out), nprocs=world,
                           join=True, start_method="spawn")
        ref = mcmc.Chains(_model(), _starts(n_total), SEED, _phi).run(STEPS)
        for r in range(world):
            d = np.load(os.path.join(out, f"rank{r}.npz"))
            assert np.array_equal(d["pooled"], ref)
            units, secs, rate = d["agg"]
            assert units == n_total * STEPS and secs == float(world) and rate == units / secs
