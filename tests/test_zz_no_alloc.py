"""rd_evaluate_batch_noalloc, the entry point for callers that cannot
allocate device memory during a call (their device memory is reserved by
another allocator, or they must not stall on cudaFree's synchronisation):
through the C ABI it must give the same results as rd_evaluate_batch, twice
in a row (its fixed scratch keeps the previous call's contents), leave the
device's free memory unchanged from before its first call on a new problem
even for a batch that rd_evaluate_batch would have to grow its workspace
for, and reject batches beyond its fixed limit.
This file is collected last so that a failure here comes after every other
test has run."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1605_04718_gb300 as rd
import rd_synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def _buffers(B, n):
    dev = torch.device("cuda:0")
    return (torch.zeros(B, dtype=torch.float64, device=dev),
            torch.zeros(B, dtype=torch.int32, device=dev),
            torch.full((B, 2, n, n), float("nan"), dtype=torch.float32, device=dev))


@pytest.mark.parametrize("solver", [rd.RD_SOLVER_DCT_TC, rd.RD_SOLVER_DCT_SIMT])
def test_noalloc_matches_evaluate_batch_twice(solver):
    dss = [H.small_dataset(n, 60, seed=500 + n) for n in (32, 64)]
    dev = torch.device("cuda:0")
    # a batch larger than a new problem's workspace (1024 work-list slots), so
    # that rd_evaluate_batch would have to grow it with cudaMalloc
    B = 4096
    theta = rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.15] * 4, B, seed=21)
    theta[3, 3] = 5e4  # one divergent proposal: NONFINITE on both paths
    th = torch.tensor(theta, dtype=torch.float64, device=dev)
    sz = torch.tensor(np.arange(B) % 2, dtype=torch.int32, device=dev)
    # load the solve kernels once on another problem, so that the driver's
    # loading of code on first launch is not counted below
    warm = H.gpu_problem(dss, solver=solver)
    pw, sw, fw = _buffers(B, 64)
    rd.rd_evaluate_batch(warm, th, pw, sw, size_idx=sz, fields=fw)
    rd.rd_sync(warm)
    rd.rd_problem_destroy(warm)
    del pw, sw, fw
    p = H.gpu_problem(dss, solver=solver)  # fresh problem: no call has run on it
    # output buffers of both calls allocated and filled beforehand: nothing but
    # the calls themselves runs between the free-memory readings
    bufs = [_buffers(B, 64) for _ in range(2)]
    results = []
    torch.cuda.synchronize(dev)
    free_before = torch.cuda.mem_get_info(dev)[0]
    for phi1, st1, fl1 in bufs:
        rd.rd_evaluate_batch_noalloc(p, th, phi1, st1, size_idx=sz, fields=fl1)
        rd.rd_sync(p)
        assert torch.cuda.mem_get_info(dev)[0] == free_before  # the call allocated nothing
    for phi1, st1, fl1 in bufs:
        results.append((phi1.cpu().numpy(), st1.cpu().numpy(), fl1.double().cpu().numpy()))
    # the existing entry point afterwards (it grows the workspace) as the reference
    phi0, st0, fl0 = _buffers(B, 64)
    rd.rd_evaluate_batch(p, th, phi0, st0, size_idx=sz, fields=fl0)
    rd.rd_sync(p)
    p0, s0, f0 = phi0.cpu().numpy(), st0.cpu().numpy(), fl0.double().cpu().numpy()
    for p1, s1, f1 in results:
        assert np.array_equal(s0, s1)
        assert s1[3] & rd.RD_P_NONFINITE
        ok = s0 == 0
        assert ok.sum() > B // 2
        assert np.all(np.abs(p1[ok] - p0[ok]) <= 1e-6 * np.abs(p0[ok]))
        assert np.all(np.isinf(p1[~ok]))
        for parity, n in ((0, 32), (1, 64)):
            idx = np.nonzero(ok & (np.arange(B) % 2 == parity))[0]
            a = f0[idx].reshape(len(idx), -1)[:, : 2 * n * n]
            b = f1[idx].reshape(len(idx), -1)[:, : 2 * n * n]
            err = np.sqrt(((b - a) ** 2).sum(1) / (a ** 2).sum(1))
            assert err.max() < 1e-6
    rd.rd_problem_destroy(p)


def test_noalloc_rejects_batches_beyond_its_limit():
    ds = H.small_dataset(16, 10, seed=7)
    p = H.gpu_problem([ds], solver=rd.RD_SOLVER_DCT_TC)
    L = rd.load()
    code = L.rd_evaluate_batch_noalloc(p, rd.RD_NOALLOC_MAX_BATCH + 1, None, None, None, None, None)
    assert code == rd.RD_EINVAL
    assert str(rd.RD_NOALLOC_MAX_BATCH) in rd.rd_last_error()
    assert L.rd_evaluate_batch_noalloc(p, 0, None, None, None, None, None) == rd.RD_OK
    rd.rd_problem_destroy(p)
