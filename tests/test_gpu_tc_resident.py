"""Parity of the 128^2 tensor-core solve whose DCT matrices stay resident in
tensor memory (RD_KERNEL_TC_RESIDENT) with the FP64 oracle, through the C
ABI.  That kernel alternates the state's orientation every step, so the
cases cover odd and even step counts, observations at odd and even steps,
the growing domain, two 128^2 datasets in one launch, and a 128^2 size next
to sizes that run the stacked kernel.  Tolerances as in test_gpu_parity:
fields within relative L2 1e-3 (FP32), Phi within what that field
tolerance allows."""
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
TC = rd.RD_SOLVER_DCT_TC
TRUE4 = [0.1, 0.9, 10.0, 200.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def _eval(p, theta, nmax, size_idx=None):
    B = theta.shape[0]
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    phi = torch.zeros(B, dtype=torch.float64, device=DEV)
    st = torch.zeros(B, dtype=torch.int32, device=DEV)
    sz = torch.tensor(size_idx, dtype=torch.int32, device=DEV) if size_idx is not None else None
    fl = torch.full((B, 2, nmax, nmax), float("nan"), dtype=torch.float32, device=DEV)
    rd.rd_evaluate_batch(p, th, phi, st, size_idx=sz, fields=fl)
    rd.rd_sync(p)
    return phi.cpu().numpy(), st.cpu().numpy().astype(np.uint32), fl.double().cpu().numpy()


def _draws(n, seed, sd=0.15):
    return rd_synth.lognormal_draws(TRUE4, [sd] * 4, n, seed)


def _oracle_all(ds, theta):
    """Oracle Phi, status, final fields and observed fields of each row."""
    P = H.oracle_problem(ds)
    th5 = theta if theta.shape[1] == 5 else np.concatenate([theta, np.zeros((len(theta), 1))], 1)
    with cf.ThreadPoolExecutor(max_workers=min(8, len(theta))) as ex:
        return list(ex.map(lambda t: P.forward(list(t), want_obs=True), th5))


def _check(ds, theta, phi, st, fl, rel_tol=1e-3):
    n = ds["n"]
    for i, (po, so, uo, vo, obs) in enumerate(_oracle_all(ds, theta)):
        assert st[i] == so, (i, st[i], so)
        if so:
            continue
        w_o = np.stack([uo, vo]).reshape(2, -1)
        w_g = fl[i].reshape(-1)[: 2 * n * n].reshape(2, -1)
        assert H.rel_l2(w_g, w_o) < rel_tol, (i, H.rel_l2(w_g, w_o))
        tol = H.phi_tolerance(ds["y"].reshape(-1), obs.reshape(-1), ds["sigma"], rel_field=rel_tol)
        assert abs(phi[i] - po) <= tol, (i, phi[i], po, tol)


def test_default_kernel_choice():
    ds = H.small_dataset(128, 4, seed=1)
    p = H.gpu_problem([ds, H.small_dataset(64, 4, seed=2)], solver=TC)
    assert rd.rd_get_size_kernel(p, 0) == rd.RD_KERNEL_TC_RESIDENT
    assert rd.rd_get_size_kernel(p, 1) == rd.RD_KERNEL_TC_STACKED
    with pytest.raises(rd.RdError):
        rd.rd_set_size_kernel(p, 1, rd.RD_KERNEL_TC_RESIDENT)  # N = 64
    with pytest.raises(rd.RdError):
        rd.rd_set_size_kernel(p, 2, rd.RD_KERNEL_SIMT)  # no such size
    with pytest.raises(rd.RdError):
        rd.rd_set_size_kernel(p, 0, 7)
    rd.rd_set_size_kernel(p, 0, rd.RD_KERNEL_SIMT)
    assert rd.rd_get_size_kernel(p, 0) == rd.RD_KERNEL_SIMT
    rd.rd_problem_destroy(p)
    p = H.gpu_problem([ds], solver=rd.RD_SOLVER_DCT_SIMT)
    assert rd.rd_get_size_kernel(p, 0) == rd.RD_KERNEL_SIMT
    rd.rd_problem_destroy(p)


@pytest.mark.parametrize("n_steps,obs_frac", [(101, (1.0,)), (100, (1.0,)), (1, (1.0,)),
                                              (75, (0.04, 0.52, 1.0))])
def test_resident_matches_oracle(n_steps, obs_frac):
    """Odd and even final steps; observations at steps of both parities
    (3, 39, 75) so both orientations are read."""
    ds = H.small_dataset(128, n_steps, seed=900 + n_steps, obs_frac=obs_frac)
    p = H.gpu_problem([ds], solver=TC)
    assert rd.rd_get_size_kernel(p, 0) == rd.RD_KERNEL_TC_RESIDENT
    theta = np.concatenate([[TRUE4], _draws(4, seed=n_steps)])
    phi, st, fl = _eval(p, theta, 128)
    _check(ds, theta, phi, st, fl)
    rd.rd_problem_destroy(p)


def test_resident_stacked_and_simt_all_match_oracle():
    """The three kernels of a 128^2 size on the same proposals: identical
    status bits, and each within the field tolerance of the oracle (two FP32
    solves may differ from each other by up to twice that)."""
    ds = H.small_dataset(128, 300, seed=31)
    theta = _draws(10, seed=32)
    p = H.gpu_problem([ds], solver=TC)
    out = {}
    for k in (rd.RD_KERNEL_TC_RESIDENT, rd.RD_KERNEL_TC_STACKED, rd.RD_KERNEL_SIMT):
        rd.rd_set_size_kernel(p, 0, k)
        out[k] = _eval(p, theta, 128)
    rd.rd_problem_destroy(p)
    for k, res in out.items():
        assert np.array_equal(res[1], out[rd.RD_KERNEL_SIMT][1])
        _check(ds, theta, *res)


def test_resident_growing_domain():
    """rho(t) = exp(r t) with r inferred: the scale factors change every step."""
    n, steps, tau = 128, 300, 1e-3
    ds = H.small_dataset(n, steps, tau=tau, seed=41, field_mask=1, obs_frac=(0.5, 1.0),
                         sigma=0.02)
    model = dict(param_map=[0, 1, 2, 3, 4],
                 prior_kind=[rd.RD_PRIOR_LOGNORMAL] * 4 + [rd.RD_PRIOR_UNIFORM],
                 prior_p0=TRUE4 + [0.0], prior_p1=[0.5] * 4 + [0.05],
                 step_space=[rd.RD_STEP_LOG] * 4 + [rd.RD_STEP_LINEAR])
    theta = np.concatenate([_draws(4, seed=42), np.linspace(0.0, 0.05, 4)[:, None]], 1)
    p = H.gpu_problem([ds], solver=TC, growth=1, model=model)
    assert rd.rd_get_size_kernel(p, 0) == rd.RD_KERNEL_TC_RESIDENT
    phi, st, fl = _eval(p, theta, n)
    rd.rd_problem_destroy(p)
    P = oracle.Problem(2, n, tau, steps, ds["u0"], ds["v0"], y=ds["y"],
                       obs_steps=ds["obs_steps"], field_mask=1, sigma=0.02)
    res = P.forward_batch(theta, want_fields=True)
    for i in range(len(theta)):
        assert st[i] == res[1][i] == 0
        assert H.rel_l2(fl[i], res[2][i]) < 1e-3, i
        assert abs(phi[i] - res[0][i]) <= 2e-3 * res[0][i] + 1.0, (i, phi[i], res[0][i])


def test_two_128_datasets_and_a_stacked_size():
    """Sizes 0 and 2 are both 128^2 (different data, one resident launch);
    size 1 is 64^2 (the stacked kernel, a second launch)."""
    dss = [H.small_dataset(128, 60, seed=51), H.small_dataset(64, 60, seed=52),
           H.small_dataset(128, 60, seed=53)]
    p = H.gpu_problem(dss, solver=TC)
    B = 13
    theta = _draws(B, seed=54)
    size_idx = np.array([0, 1, 2] * 4 + [2])
    phi, st, fl = _eval(p, theta, 128, size_idx=size_idx)
    rd.rd_problem_destroy(p)
    for s, ds in enumerate(dss):
        idx = np.nonzero(size_idx == s)[0]
        n = ds["n"]
        sub = np.stack([fl[i].reshape(-1)[: 2 * n * n] for i in idx]).reshape(len(idx), 2, n, n)
        _check(ds, theta[idx], phi[idx], st[idx], sub)


def test_resident_full_size_sampled_outputs():
    """The benchmark's launch: 4096 proposals of the stored 128^2 dataset,
    8000 steps; sampled rows against the oracle."""
    ds = H.stored_2d("rd2d_n128")
    B = 4096
    p = H.gpu_problem([ds], solver=rd.RD_SOLVER_AUTO)
    assert rd.rd_get_size_kernel(p, 0) == rd.RD_KERNEL_TC_RESIDENT
    theta = _draws(B, seed=78)
    theta[0] = TRUE4
    phi, st, fl = _eval(p, theta, 128)
    rd.rd_problem_destroy(p)
    pick = [0, 3, B // 3, B - 2]
    P = H.oracle_problem(ds)
    with cf.ThreadPoolExecutor(max_workers=len(pick)) as ex:
        outs = list(ex.map(lambda t: P.forward(list(t) + [0.0]), theta[pick]))
    for i, (po, so, uo, vo) in zip(pick, outs):
        assert st[i] == so
        if so:
            continue
        w_o = np.stack([uo, vo])
        assert H.rel_l2(fl[i], w_o) < 1e-3, (i, H.rel_l2(fl[i], w_o))
        assert abs(phi[i] - po) <= H.phi_tolerance(ds["y"].reshape(2, -1), w_o.reshape(2, -1),
                                                   ds["sigma"])
    ok = st == 0
    assert ok.mean() > 0.9 and np.all(np.isfinite(phi[ok]))
