"""Failure detection of the tensor-core solve kernels, tested without a GPU
fault: a test aid makes the MMA-issuing warp wait on a barrier that nothing
completes, the problem's wait limit is set short, and the launch must end in
bounded time with RD_ETIMEOUT, every proposal left RD_P_NOT_SOLVED with
Phi = +inf, and the problem still usable: the next normal launch (which
allocates the tensor memory the failed CTAs had to free) gives the results
of a launch before the failure."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1605_04718_gb300 as rd
import rd_synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
TRUE4 = [0.1, 0.9, 10.0, 200.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def _eval(p, th):
    B = th.shape[0]
    phi = torch.full((B,), -1.0, dtype=torch.float64, device=DEV)
    st = torch.full((B,), -1, dtype=torch.int32, device=DEV)
    rd.rd_evaluate_batch(p, th, phi, st)
    return phi, st


@pytest.mark.parametrize("n,kernel", [(128, rd.RD_KERNEL_TC_RESIDENT),
                                      (64, rd.RD_KERNEL_TC_STACKED)])
def test_bounded_wait_gives_up_and_problem_recovers(n, kernel):
    ds = H.small_dataset(n, 6, seed=900 + n)
    p = H.gpu_problem([ds], solver=rd.RD_SOLVER_DCT_TC)
    rd.rd_set_size_kernel(p, 0, kernel)
    B = 400  # more proposals than CTAs: some are never popped
    theta = rd_synth.lognormal_draws(TRUE4, [0.1] * 4, B, seed=31)
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    phi0, st0 = _eval(p, th)
    rd.rd_sync(p)
    st0 = st0.cpu().numpy()
    assert np.all(st0 == 0)

    rd.rd_set_wait_limit(p, 0.05)
    rd.rd_debug_stall_at_step(p, 2)
    t0 = time.perf_counter()
    phi1, st1 = _eval(p, th)
    with pytest.raises(rd.RdError) as ei:
        rd.rd_sync(p)
    assert ei.value.code == rd.RD_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert np.all(st1.cpu().numpy() == rd.RD_P_NOT_SOLVED)
    assert np.all(np.isinf(phi1.cpu().numpy()))
    rd.rd_sync(p)  # the flag was cleared by the report
    # the host-buffer call reports the same failure
    with pytest.raises(rd.RdError) as ei:
        rd.rd_evaluate_batch_host(p, theta)
    assert ei.value.code == rd.RD_ETIMEOUT

    rd.rd_debug_stall_at_step(p, -1)
    rd.rd_set_wait_limit(p, 4.0)
    phi2, st2 = _eval(p, th)
    rd.rd_sync(p)
    assert np.array_equal(st2.cpu().numpy(), st0)
    a, b = phi2.cpu().numpy(), phi0.cpu().numpy()
    assert np.all(np.abs(a - b) <= 1e-12 * np.abs(b))
    with pytest.raises(rd.RdError):
        rd.rd_set_wait_limit(p, 0.0)
    rd.rd_problem_destroy(p)


def test_failed_chain_step_rejects_every_unsolved_proposal():
    """A chain step whose solves gave up moves no chain: unsolved proposals
    carry RD_P_NOT_SOLVED, which the accept step rejects."""
    ds = H.small_dataset(64, 6, seed=77)
    p = H.gpu_problem([ds], solver=rd.RD_SOLVER_DCT_TC)
    C = 64
    theta0 = rd_synth.chain_starts(TRUE4, C, seed=5, rel=0.01)
    c = rd.rd_chains_create(p, theta0, 11, [0.01] * 4, capacity=4)
    th_before, phi_before = rd.rd_chains_get_state(c, 4, C)
    rd.rd_set_wait_limit(p, 0.05)
    rd.rd_debug_stall_at_step(p, 1)
    rd.rd_chains_run(c, 1)
    with pytest.raises(rd.RdError) as ei:
        rd.rd_sync(p)
    assert ei.value.code == rd.RD_ETIMEOUT
    th_after, phi_after = rd.rd_chains_get_state(c, 4, C)
    assert np.array_equal(th_after, th_before)
    assert np.array_equal(phi_after, phi_before)
    rd.rd_debug_stall_at_step(p, -1)
    rd.rd_set_wait_limit(p, 4.0)
    rd.rd_chains_run(c, 1)
    rd.rd_sync(p)
    smp, cnt = rd.rd_chains_read_samples(c, 4, 4, C)
    assert cnt[0] == 2 * C and cnt[2] > 0  # the second step accepted some proposals
    rd.rd_chains_destroy(c)
    rd.rd_problem_destroy(p)
