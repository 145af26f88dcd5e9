"""Uneven batching with per-size kernels chosen by the timed search, through
the C ABI: rd_autotune's times and choice, parity of a mixed 32^2 / 64^2 /
128^2 batch with the oracle under the tuned kernels, and the persisted table
being reused."""
import numpy as np
import pytest
import torch

import oracle
import paper_1605_04718_gb300 as rd
from paper_1605_04718_gb300 import autotune as at
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


def _draws(n, seed):
    return rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.15] * 4, n, seed)


def test_autotune_times_and_choice():
    dss = [H.small_dataset(n, 40, seed=600 + n) for n in (32, 64, 128)]
    p = H.gpu_problem(dss, solver=rd.RD_SOLVER_AUTO)
    times = rd.rd_autotune(p, _draws(64, 1), n_trials=2, probe_steps=20, n_sizes=3)
    assert times.shape == (3, 4)
    assert np.all(np.isnan(times[:, 3]))  # CG needs every grid at N <= 96
    assert np.all(np.isfinite(times[:, :2])) and np.all(times[:, :2] > 0)
    assert np.isnan(times[0, 2]) and np.isnan(times[1, 2]) and np.isfinite(times[2, 2])
    for s in range(3):
        assert rd.rd_get_size_kernel(p, s) == at.fastest(times[s])
        assert rd.rd_get_size_schedule(p, s) >= 1  # the searched CTAs-per-SM axis
    # the tuned kernels solve a mixed batch like the oracle
    B = 24
    theta = _draws(B, 2)
    size_idx = np.arange(B) % 3
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    phi = torch.zeros(B, dtype=torch.float64, device=DEV)
    st = torch.zeros(B, dtype=torch.int32, device=DEV)
    fl = torch.zeros((B, 2, 128, 128), dtype=torch.float32, device=DEV)
    rd.rd_evaluate_batch(p, th, phi, st, size_idx=torch.tensor(size_idx, dtype=torch.int32,
                                                                device=DEV), fields=fl)
    rd.rd_sync(p)
    rd.rd_problem_destroy(p)
    phi, st, fl = phi.cpu().numpy(), st.cpu().numpy(), fl.double().cpu().numpy()
    for s, ds in enumerate(dss):
        n = ds["n"]
        P = H.oracle_problem(ds)
        for i in np.nonzero(size_idx == s)[0]:
            po, so, uo, vo = P.forward(list(theta[i]) + [0.0])
            assert st[i] == so
            w_g = fl[i].reshape(-1)[: 2 * n * n].reshape(2, -1)
            w_o = np.stack([uo, vo]).reshape(2, -1)
            assert H.rel_l2(w_g, w_o) < 1e-3
            assert abs(phi[i] - po) <= H.phi_tolerance(ds["y"].reshape(-1), w_o.reshape(-1),
                                                       ds["sigma"])


def test_tune_persists_and_reuses(tmp_path, monkeypatch):
    dss = [H.small_dataset(n, 20, seed=700 + n) for n in (64, 128)]
    p = H.gpu_problem(dss, solver=rd.RD_SOLVER_AUTO)
    path = str(tmp_path / "kernels.json")
    gpu = torch.cuda.get_device_name(0)
    first = at.tune(p, gpu, 2, [64, 128], 20, _draws(32, 3), cache_path=path, n_trials=1,
                    probe_steps=10)
    assert not first[0]["cached"]
    chosen = [rd.rd_get_size_kernel(p, s) for s in (0, 1)]
    rd.rd_problem_destroy(p)

    def no_timing(*a, **k):
        raise AssertionError("the persisted table should have been used")

    monkeypatch.setattr(at, "rd_autotune", no_timing)
    p = H.gpu_problem(dss, solver=rd.RD_SOLVER_AUTO)
    again = at.tune(p, gpu, 2, [64, 128], 20, _draws(32, 3), cache_path=path)
    assert again[0]["cached"] and again[1]["cached"]
    assert [rd.rd_get_size_kernel(p, s) for s in (0, 1)] == chosen
    rd.rd_problem_destroy(p)
