"""The evolving-domain workload at its full size, through the C ABI: the
stored 128^2 dataset on a growing square rho(t) = exp(r t) (tau = 1e-4,
50000 IMEX steps to T = 5, u observed at 5 times, sigma = 0.02), 2048
proposals with r inferred, in one launch of the library's default kernel for
the size.  Sampled rows are compared with the FP64 oracle (fields within
relative L2 1e-3, Phi within what that field tolerance allows); every row's
status and finiteness is checked."""
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
MODEL5 = dict(param_map=[0, 1, 2, 3, 4],
              prior_kind=[rd.RD_PRIOR_LOGNORMAL] * 4 + [rd.RD_PRIOR_UNIFORM],
              prior_p0=[0.1, 0.9, 10.0, 200.0, 0.0], prior_p1=[0.5] * 4 + [0.05],
              step_space=[rd.RD_STEP_LOG] * 4 + [rd.RD_STEP_LINEAR])


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def test_growing_domain_full_size_sampled_outputs():
    ds = H.stored_2d("rd2d_n128_grow")
    n, B = ds["n"], 2048
    p = H.gpu_problem([ds], solver=rd.RD_SOLVER_AUTO, growth=1, model=MODEL5)
    theta = np.concatenate([rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.1] * 4, B, 91),
                            rd_synth.uniform_draws([0.0], [0.02], B, 92)], 1)
    theta[0] = [0.1, 0.9, 10.0, 200.0, 0.01]
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    phi = torch.zeros(B, dtype=torch.float64, device=DEV)
    st = torch.zeros(B, dtype=torch.int32, device=DEV)
    fl = torch.zeros((B, 2, n, n), dtype=torch.float32, device=DEV)
    rd.rd_evaluate_batch(p, th, phi, st, fields=fl)
    rd.rd_sync(p)
    rd.rd_problem_destroy(p)
    phi, st = phi.cpu().numpy(), st.cpu().numpy().astype(np.uint32)
    pick = [0, B // 2 + 7]
    P = oracle.Problem(2, n, ds["tau"], ds["n_steps"], ds["u0"], ds["v0"], y=ds["y"],
                       obs_steps=ds["obs_steps"], field_mask=1, sigma=ds["sigma"])
    with cf.ThreadPoolExecutor(max_workers=len(pick)) as ex:
        outs = list(ex.map(lambda t: P.forward(list(t), want_obs=True), theta[pick]))
    for i, (po, so, uo, vo, obs) in zip(pick, outs):
        assert st[i] == so
        if so:
            continue
        w_o = np.stack([uo, vo])
        w_g = fl[i].double().cpu().numpy()
        assert H.rel_l2(w_g, w_o) < 1e-3, (i, H.rel_l2(w_g, w_o))
        tol = H.phi_tolerance(ds["y"].reshape(-1), obs.reshape(-1), ds["sigma"])
        assert abs(phi[i] - po) <= tol, (i, phi[i], po, tol)
    ok = st == 0
    assert ok.mean() > 0.9 and np.all(np.isfinite(phi[ok]))
