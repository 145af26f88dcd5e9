"""The uneven batch at its full size, through the C ABI: the stored 64^2,
96^2 and 128^2 datasets (8000 IMEX steps each) as three grid sizes of one
problem, 4096 proposals with a third of each size interleaved, in the
library's default per-size kernels (one persistent launch per kernel kind).
One sampled proposal of each size is compared with the FP64 oracle (fields
within relative L2 1e-3, Phi within what that allows); every status and Phi
is checked for finiteness."""
import concurrent.futures as cf

import numpy as np
import pytest
import torch

import oracle
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


def test_mixed_sizes_full_size_sampled_outputs():
    dss = [H.stored_2d(nm) for nm in ("rd2d_n64", "rd2d_n96", "rd2d_n128")]
    p = H.gpu_problem(dss, solver=rd.RD_SOLVER_AUTO)
    B = 4096
    theta = rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.15] * 4, B, 95)
    size_idx = np.arange(B) % 3
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    phi = torch.zeros(B, dtype=torch.float64, device=DEV)
    st = torch.zeros(B, dtype=torch.int32, device=DEV)
    fl = torch.zeros((B, 2, 128, 128), dtype=torch.float32, device=DEV)
    rd.rd_evaluate_batch(p, th, phi, st, size_idx=torch.tensor(size_idx, dtype=torch.int32,
                                                                device=DEV), fields=fl)
    rd.rd_sync(p)
    rd.rd_problem_destroy(p)
    phi, st = phi.cpu().numpy(), st.cpu().numpy().astype(np.uint32)
    pick = [3 * 700, 3 * 900 + 1, 3 * 1100 + 2]  # one proposal of each size
    assert [size_idx[i] for i in pick] == [0, 1, 2]

    def run(i):
        ds = dss[size_idx[i]]
        return H.oracle_problem(ds).forward(list(theta[i]) + [0.0])

    with cf.ThreadPoolExecutor(max_workers=3) as ex:
        outs = list(ex.map(run, pick))
    for i, (po, so, uo, vo) in zip(pick, outs):
        ds = dss[size_idx[i]]
        n = ds["n"]
        assert st[i] == so
        if so:
            continue
        w_o = np.stack([uo, vo]).reshape(2, -1)
        w_g = fl[i].reshape(-1)[: 2 * n * n].reshape(2, -1).double().cpu().numpy()
        assert H.rel_l2(w_g, w_o) < 1e-3, (i, n, H.rel_l2(w_g, w_o))
        assert abs(phi[i] - po) <= H.phi_tolerance(ds["y"].reshape(2, -1), w_o, ds["sigma"])
    ok = st == 0
    assert ok.mean() > 0.9 and np.all(np.isfinite(phi[ok]))
    for s in range(3):
        assert np.all(np.isfinite(phi[(size_idx == s) & ok]))
