"""The learned surrogate on the GPU (hand-written BF16 tcgen05 GEMMs) against
the FP64 oracle network, and delayed-acceptance chains against the oracle's
delayed-acceptance sampler.

Tolerances: with the oracle evaluating the network at the kernels' BF16
rounding points, loss within 1e-4 relative and every gradient block within
relative L2 2e-3 (FP32 accumulation order and fast exp in SiLU differ); against
the plain FP64 network, gradients within relative L2 5e-2 (BF16 rounding of
weights and activations, 2^-8 per element).  Posteriors of the delayed-
acceptance chains: means and 95% interval ends within 3 bootstrap standard
errors (resampling independent chains) of the oracle's and of plain chains."""
import numpy as np
import pytest
import torch

import oracle
import paper_1605_04718_gb300 as rd
import rd_synth
from oracle import mcmc, mlp
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
W = rd.RD_SURROGATE_WIDTH


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_04718_gb300 import build
    build.build()
    oracle.build()
    rd.load()


def _problem():
    ds = H.small_dataset(16, 20, seed=1)
    return H.gpu_problem([ds]), ds


def _random_params(seed):
    params = mlp.init_params((mlp.N_IN, W, W, W, 1), seed)
    rng = np.random.default_rng(seed + 100)
    for layer in params:
        layer[1] += rng.normal(0, 0.05, layer[1].shape)
    params[0][0][:, 4:] = 0.0  # padded inputs
    params[-1][0] *= 5.0
    return params


def _norm(mu, sd, floor=10.0, shift=2.0, scale=0.5):
    n = np.zeros(2 * rd.RD_NPARAM + 3)
    n[:4], n[5:9] = mu, sd
    n[4], n[9] = 0.0, 1.0
    n[10:] = [floor, shift, scale]
    return n


def _features(theta, norm):
    x = np.zeros((theta.shape[0], mlp.N_IN))
    x[:, :4] = (np.log(theta) - norm[:4]) / norm[5:9]
    return x


def test_mlp_loss_and_gradients_match_oracle():
    p, _ = _problem()
    s = rd.rd_surrogate_create(p, seed=1)
    params = _random_params(7)
    norm = _norm(np.log([0.1, 0.9, 10.0, 200.0]), [0.5] * 4)
    rd.rd_surrogate_set_params(s, mlp.flatten(params).astype(np.float32), norm)
    B = 384
    theta = rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.5] * 4, B, seed=3)
    target = np.random.default_rng(4).standard_normal(B).astype(np.float32)
    grads = torch.zeros(mlp.flat_layout(W)[1], dtype=torch.float32, device=DEV)
    loss = rd.rd_surrogate_loss_grad(
        s, torch.tensor(theta, device=DEV), torch.tensor(target, device=DEV), grads)
    g_gpu = grads.double().cpu().numpy()
    # the oracle at the kernels' precision (parameters as the GPU stores them: FP32)
    p32 = mlp.unflatten(mlp.flatten(params).astype(np.float32), W)
    x = _features(theta, norm)
    l_ref, g_ref, _ = mlp.loss_and_grads_bf16(p32, x, target.astype(np.float64))
    assert loss == pytest.approx(l_ref, rel=1e-4)
    lay, _ = mlp.flat_layout(W)
    flat_ref = mlp.flatten(g_ref)
    for name, (off, shp) in lay.items():
        n = int(np.prod(shp))
        a, b = g_gpu[off:off + n], flat_ref[off:off + n]
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b) + 1e-12, name
    # and against the plain FP64 network
    l64, g64 = mlp.loss_and_grads(p32, x, target.astype(np.float64))
    flat64 = mlp.flatten(g64)
    assert loss == pytest.approx(l64, rel=2e-2)
    assert np.linalg.norm(g_gpu - flat64) <= 5e-2 * np.linalg.norm(flat64)
    rd.rd_surrogate_destroy(s)
    rd.rd_problem_destroy(p)


def test_mlp_predict_matches_oracle():
    p, _ = _problem()
    s = rd.rd_surrogate_create(p, seed=2)
    params = _random_params(8)
    norm = _norm(np.log([0.1, 0.9, 10.0, 200.0]), [0.5] * 4, floor=100.0, shift=3.0, scale=0.7)
    rd.rd_surrogate_set_params(s, mlp.flatten(params).astype(np.float32), norm)
    B = 1000  # not a multiple of 128: ragged last tile
    theta = rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.5] * 4, B, seed=5)
    out = torch.zeros(B, dtype=torch.float64, device=DEV)
    rd.rd_surrogate_predict(s, torch.tensor(theta, device=DEV), out)
    torch.cuda.synchronize()
    p32 = mlp.unflatten(mlp.flatten(params).astype(np.float32), W)
    _, _, net = mlp.loss_and_grads_bf16(p32, _features(theta, norm), np.zeros(B))
    ref = norm[10] + np.exp(norm[11] + norm[12] * net)
    got = out.cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-4)
    rd.rd_surrogate_destroy(s)
    rd.rd_problem_destroy(p)


def test_training_learns_a_smooth_log_likelihood():
    """Phi = 500 + 2000 sum_j (log theta_j - log m_j)^2 on prior draws: after
    training the hold-out relative error of Phi~ is small."""
    p, _ = _problem()
    s = rd.rd_surrogate_create(p, seed=3)
    n = 16384
    med = np.array([0.1, 0.9, 10.0, 200.0])
    theta = rd_synth.lognormal_draws(med, [0.5] * 4, n, seed=9)
    phi = 500.0 + 2000.0 * ((np.log(theta) - np.log(med)) ** 2).sum(1)
    rep = rd.rd_surrogate_train(s, torch.tensor(theta, device=DEV), torch.tensor(phi, device=DEV),
                                epochs=40, batch=512, lr=2e-3, holdout_frac=0.1, seed=1)
    assert np.all(np.isfinite(rep))
    assert rep[1] < 0.02 and rep[2] < 0.05, rep
    params, norm = rd.rd_surrogate_get_params(s)
    assert norm[10] == pytest.approx(phi.min() - 1.0)
    rd.rd_surrogate_destroy(s)
    rd.rd_problem_destroy(p)


def _oracle_surrogate(ds, P_or, seed=0, n=1536, epochs=150):
    """An FP64 surrogate trained by the oracle on oracle (theta, Phi) pairs
    drawn around the truth; returns (flat params, norm, phi_tilde function)."""
    theta = rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.03] * 4, n, seed=seed)
    phi, st = P_or.forward_batch(np.concatenate([theta, np.zeros((n, 1))], 1))
    ok = (st == 0) & np.isfinite(phi)
    theta, phi = theta[ok], phi[ok]
    norm = np.zeros(2 * rd.RD_NPARAM + 3)
    lt = np.log(theta)
    norm[:4], norm[5:9] = lt.mean(0), lt.std(0)
    norm[9] = 1.0
    floor = phi.min() - 1.0
    z = np.log(phi - floor)
    norm[10:] = [floor, z.mean(), z.std()]
    x = _features(theta, norm)
    target = (z - norm[11]) / norm[12]
    params = mlp.init_params((mlp.N_IN, W, W, W, 1), seed)
    params[0][0][:, 4:] = 0.0
    opt = mlp.Adam(params, lr=1e-3)
    for _ in range(epochs):
        _, g = mlp.loss_and_grads(params, x, target)
        opt.step(params, g)
    flat = mlp.flatten(params).astype(np.float32)
    p32 = mlp.unflatten(flat, W)

    def phit(th):
        out, _ = mlp.forward(p32, _features(np.atleast_2d(th), norm))
        return norm[10] + np.exp(norm[11] + norm[12] * out)

    return flat, norm, phit


def _boot_se(a, b, stat, n_boot=300, seed=0):
    """Standard error of stat(a) - stat(b) for pooled samples [steps][chains]
    of independent chains, by resampling chains."""
    rng = np.random.default_rng(seed)
    ca, cb = a.shape[1], b.shape[1]
    d = [stat(a[:, rng.integers(0, ca, ca)]) - stat(b[:, rng.integers(0, cb, cb)])
         for _ in range(n_boot)]
    return float(np.std(d))


def test_delayed_acceptance_chains_match_oracle_posterior():
    """Delayed acceptance with an oracle-trained surrogate: the GPU chains, the
    oracle's delayed-acceptance chains and plain GPU chains, all started from
    states the oracle's own plain sampler burned in, agree in posterior mean
    and 95% interval ends within 3 bootstrap standard errors (chains are
    independent, so resampling chains gives honest errors)."""
    ds = H.small_dataset(16, 100, seed=9, sigma=0.05)
    P_or = H.oracle_problem(ds)
    flat, norm, phit = _oracle_surrogate(ds, P_or)
    C, S = 64, 600
    step = [0.02, 0.02, 0.05, 0.05]
    m = mcmc.Model([0, 1, 2, 3], np.array([0.1, 0.9, 10.0, 200.0, 0.0]), ["lognormal"] * 4,
                   np.array([0.1, 0.9, 10.0, 200.0]), np.array([0.5] * 4), ["log"] * 4,
                   np.asarray(step))
    burn = mcmc.Chains(m, rd_synth.chain_starts([0.1, 0.9, 10.0, 200.0], C, seed=200), 5,
                       lambda th: P_or.forward_batch(th))
    burn.run(400)
    theta0 = burn.theta.copy()
    p = H.gpu_problem([ds])
    s = rd.rd_surrogate_create(p, seed=4)
    rd.rd_surrogate_set_params(s, flat, norm)
    c = rd.rd_chains_create(p, theta0, 99, step, capacity=S)
    rd.rd_chains_set_surrogate(c, s)
    rd.rd_chains_run(c, S)
    s_da, counters = rd.rd_chains_read_samples(c, S, 4, C)
    assert counters[0] == C * S
    assert counters[3] == counters[1] < counters[0]  # only stage-1 survivors were solved
    ch = mcmc.Chains(m, theta0, 99, lambda th: P_or.forward_batch(th), surrogate=phit)
    s_orc = ch.run(S)
    c2 = rd.rd_chains_create(p, theta0, 77, step, capacity=S)
    rd.rd_chains_run(c2, S)
    s_plain, _ = rd.rd_chains_read_samples(c2, S, 4, C)
    stats = [np.mean, lambda a: np.quantile(a, 0.025), lambda a: np.quantile(a, 0.975)]
    for other in (s_orc, s_plain):
        for j in range(4):
            a, b = s_da[:, j, :], other[:, j, :]
            for stat in stats:
                se = _boot_se(a, b, stat)
                assert abs(stat(a) - stat(b)) < 3 * se + 1e-12, (j, stat(a), stat(b), se)
    for h in (c, c2):
        rd.rd_chains_destroy(h)
    rd.rd_surrogate_destroy(s)
    rd.rd_problem_destroy(p)


def test_trained_surrogate_cuts_exact_solves_per_effective_sample():
    """What the learned part gains: a surrogate trained on the GPU by the
    library's own kernels, on (theta, Phi) pairs the batched solver produced,
    screens delayed-acceptance proposals so that the exact solves spent per
    effective sample fall well below plain Metropolis' (one solve per
    proposal), while both samplers reach the same posterior: means and 95%
    interval ends within 3 combined Monte Carlo standard errors."""
    from paper_1605_04718_gb300 import stats
    ds = H.small_dataset(32, 100, seed=13, sigma=0.05)
    p = H.gpu_problem([ds], solver=rd.RD_SOLVER_DCT_TC)
    C = 128
    theta0 = rd_synth.chain_starts([0.1, 0.9, 10.0, 200.0], C, seed=31)
    step = np.array([0.02, 0.01, 0.05, 0.05])
    # pilot: burn in with plain chains, then a proposal covariance from them
    c = rd.rd_chains_create(p, theta0, 5, step, capacity=400)
    rd.rd_chains_run(c, 400)
    pilot, _ = rd.rd_chains_read_samples(c, 400, 4, C)
    start, _ = rd.rd_chains_get_state(c, 4, C)
    rd.rd_chains_destroy(c)
    lt = np.log(pilot[200:]).transpose(1, 0, 2).reshape(4, -1)
    mu, cov = lt.mean(1), np.cov(lt)
    prop = np.linalg.cholesky(2.38 ** 2 / 4 * cov)
    # training pairs from the batched exact solver, 2.5 posterior sd around it
    n = 4096
    th_tr = np.exp(mu[None, :] + 2.5 * np.random.default_rng(3).standard_normal((n, 4))
                   @ np.linalg.cholesky(cov).T)
    th_d = torch.tensor(th_tr, dtype=torch.float64, device=DEV)
    phi_d = torch.zeros(n, dtype=torch.float64, device=DEV)
    st_d = torch.zeros(n, dtype=torch.int32, device=DEV)
    rd.rd_evaluate_batch(p, th_d, phi_d, st_d)
    rd.rd_sync(p)
    s = rd.rd_surrogate_create(p, seed=6)
    rep = rd.rd_surrogate_train(s, th_d, phi_d, epochs=80, batch=512, lr=1e-3,
                                holdout_frac=0.1, seed=2)
    assert np.all(np.isfinite(rep))
    S = 1200
    out = {}
    for mode in ("plain", "da"):
        c = rd.rd_chains_create(p, start, 4242, step, capacity=S)
        rd.rd_chains_set_proposal(c, prop)
        if mode == "da":
            rd.rd_chains_set_surrogate(c, s)
        rd.rd_chains_run(c, S)
        smp, cnt = rd.rd_chains_read_samples(c, S, 4, C)
        rd.rd_chains_destroy(c)
        summ = stats.summarize(smp, burn_frac=0.25)
        ess = min(x["ess"] for x in summ)
        out[mode] = (summ, cnt[3] * 0.75 / ess, cnt)
    assert out["plain"][2][3] == out["plain"][2][0]  # plain: one solve per proposal
    assert out["da"][2][3] < 0.6 * out["da"][2][0]    # DA: only stage-1 survivors
    # exact solves per effective sample
    assert out["da"][1] < 0.7 * out["plain"][1], (out["da"][1], out["plain"][1])
    for a, b in zip(out["da"][0], out["plain"][0]):
        assert abs(a["mean"] - b["mean"]) < 3 * np.hypot(a["mcse"], b["mcse"]), (a, b)
        assert abs(a["q025"] - b["q025"]) < 3 * np.hypot(a["mcse_q025"], b["mcse_q025"]), (a, b)
        assert abs(a["q975"] - b["q975"]) < 3 * np.hypot(a["mcse_q975"], b["mcse_q975"]), (a, b)
    rd.rd_surrogate_destroy(s)
    rd.rd_problem_destroy(p)
