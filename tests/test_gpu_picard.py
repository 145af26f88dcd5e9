"""The paper's semi-implicit time step (Sec. 3.1.1, Example 1) on the GPU,
through the C ABI, against the FP64 oracle: 1-D fields and Phi on a fixed and
on a growing domain, chains with the same random streams, and the argument
checks; in 2-D (preconditioned CG on the CUDA cores) fields and Phi on two
grid sizes, the paper's gamma = 1000 setting and its fixed steady state; and
the plain-CG IMEX kernel (RD_KERNEL_CG) against the oracle."""
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
    ds2 = H.small_dataset(96, 4, seed=3)
    p2 = H.gpu_problem([ds2])
    with pytest.raises(rd.RdError):
        rd.rd_set_scheme(p2, rd.RD_SCHEME_PICARD)  # 2-D: grids up to 80 only
    rd.rd_problem_destroy(p2)


# ---- 2-D: preconditioned CG on the CUDA cores ------------------------------

def _picard2d(dss, theta, fixed=None):
    """GPU and oracle results of the semi-implicit step for proposals theta
    (natural units, [B][4]) on the 2-D datasets dss (size i % len(dss))."""
    p = H.gpu_problem(dss, solver=rd.RD_SOLVER_AUTO, fixed=fixed)
    rd.rd_set_scheme(p, rd.RD_SCHEME_PICARD)
    B = theta.shape[0]
    nmax = max(d["n"] for d in dss)
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    sz = torch.tensor(np.arange(B) % len(dss), dtype=torch.int32, device=DEV)
    phi = torch.zeros(B, dtype=torch.float64, device=DEV)
    st = torch.zeros(B, dtype=torch.int32, device=DEV)
    fl = torch.full((B, 2, nmax, nmax), float("nan"), dtype=torch.float32, device=DEV)
    rd.rd_evaluate_batch(p, th, phi, st, size_idx=sz, fields=fl)
    rd.rd_sync(p)
    rd.rd_problem_destroy(p)
    return phi.cpu().numpy(), st.cpu().numpy(), fl.double().cpu().numpy()


def _oracle2d(ds, theta):
    P = oracle.Problem(2, ds["n"], ds["tau"], ds["n_steps"], ds["u0"], ds["v0"], y=ds["y"],
                       obs_steps=ds["obs_steps"], field_mask=ds["field_mask"],
                       sigma=ds["sigma"], scheme="picard")
    th5 = np.concatenate([theta, np.zeros((len(theta), 1))], 1)
    return P.forward_batch(th5, want_fields=True)


def test_picard_2d_fields_and_phi_match_oracle():
    """Two grid sizes in one launch, prior draws around the truth, 200
    steps: fields within relative L2 1e-3 (FP32) of the FP64 oracle's CG
    solution, Phi within what that allows."""
    dss = [H.small_dataset(n, 200, seed=60 + n) for n in (32, 64)]
    B = 24
    theta = rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.15] * 4, B, seed=17)
    phi, st, fl = _picard2d(dss, theta)
    for s, ds in enumerate(dss):
        n = ds["n"]
        rows = np.arange(B)[np.arange(B) % 2 == s]
        po, so, fo = _oracle2d(ds, theta[rows])
        for k, i in enumerate(rows):
            assert st[i] == so[k]
            if so[k]:
                continue
            w_g = fl[i].reshape(-1)[: 2 * n * n].reshape(2, -1)
            w_o = fo[k].reshape(2, -1)
            assert H.rel_l2(w_g, w_o) < 1e-3, (i, H.rel_l2(w_g, w_o))
            tol = H.phi_tolerance(ds["y"].reshape(-1), w_o.reshape(-1), ds["sigma"])
            assert abs(phi[i] - po[k]) <= tol, (i, phi[i], po[k], tol)


def test_picard_2d_paper_parameters_and_steady_state():
    """The paper's Example-2 setting (gamma = 1000, tau = 1e-4, Table 1's a,
    b): a pattern grows from the perturbed steady state in step with the
    oracle; from the exact homogeneous steady state nothing moves."""
    a, b = 0.126779, 0.792366
    us, vs = oracle.steady_state(a, b)
    n = 64
    ds = H.small_dataset(n, 400, tau=1e-4, seed=71)
    ds = dict(ds, u0=ds["u0"] - 1.0 + us, v0=ds["v0"] - 0.9 + vs)  # (a, b)'s steady state
    flat = dict(ds, u0=np.full((n, n), us), v0=np.full((n, n), vs))
    theta = np.array([[a, b, 10.0, 1000.0]])
    for d_ in (ds, flat):
        phi, st, fl = _picard2d([d_], theta)
        po, so, fo = _oracle2d(d_, theta)
        assert st[0] == so[0] == 0
        w_g = fl[0].reshape(2, -1)
        assert H.rel_l2(w_g, fo[0].reshape(2, -1)) < 1e-3
        if d_ is flat:
            assert np.max(np.abs(w_g[0] - us)) < 1e-5 and np.max(np.abs(w_g[1] - vs)) < 1e-5


def test_cg_kernel_matches_oracle():
    """RD_KERNEL_CG (the IMEX step with each implicit system solved by plain
    CG) on 32^2, 64^2 and 96^2 in one launch, against the oracle's eigenbasis
    solve: fields within relative L2 1e-3, Phi within what that allows."""
    dss = [H.small_dataset(n, 100, seed=80 + n) for n in (32, 64, 96)]
    p = H.gpu_problem(dss, solver=rd.RD_SOLVER_AUTO)
    for s in range(3):
        rd.rd_set_size_kernel(p, s, rd.RD_KERNEL_CG)
    assert rd.rd_get_size_kernel(p, 2) == rd.RD_KERNEL_CG
    B = 18
    theta = rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.15] * 4, B, seed=19)
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    sz = torch.tensor(np.arange(B) % 3, dtype=torch.int32, device=DEV)
    phi = torch.zeros(B, dtype=torch.float64, device=DEV)
    st = torch.zeros(B, dtype=torch.int32, device=DEV)
    fl = torch.full((B, 2, 96, 96), float("nan"), dtype=torch.float32, device=DEV)
    rd.rd_evaluate_batch(p, th, phi, st, size_idx=sz, fields=fl)
    rd.rd_sync(p)
    phi, st, fl = phi.cpu().numpy(), st.cpu().numpy(), fl.double().cpu().numpy()
    for s, ds in enumerate(dss):
        n = ds["n"]
        P = H.oracle_problem(ds)
        for i in np.arange(B)[np.arange(B) % 3 == s]:
            po, so, uo, vo = P.forward(list(theta[i]) + [0.0])
            assert st[i] == so
            if so:
                continue
            w_g = fl[i].reshape(-1)[: 2 * n * n].reshape(2, -1)
            w_o = np.stack([uo, vo]).reshape(2, -1)
            assert H.rel_l2(w_g, w_o) < 1e-3, (i, H.rel_l2(w_g, w_o))
            tol = H.phi_tolerance(ds["y"].reshape(-1), w_o.reshape(-1), ds["sigma"])
            assert abs(phi[i] - po) <= tol
    with pytest.raises(rd.RdError):  # a 128^2 grid is beyond its shared memory
        p2 = H.gpu_problem([H.small_dataset(128, 4, seed=2)], solver=rd.RD_SOLVER_AUTO)
        try:
            rd.rd_set_size_kernel(p2, 0, rd.RD_KERNEL_CG)
        finally:
            rd.rd_problem_destroy(p2)
    rd.rd_problem_destroy(p)
