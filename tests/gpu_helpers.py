"""Shared set-up for the GPU tests: build a problem from a stored synthetic
dataset on both sides (the CUDA library through its C ABI, the oracle on the
host) with the same inputs."""
import os

import numpy as np

import oracle
import paper_1605_04718_gb300 as rd
import rd_synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

LOGN4 = dict(param_map=[0, 1, 2, 3], prior_kind=[rd.RD_PRIOR_LOGNORMAL] * 4,
             prior_p0=[0.1, 0.9, 10.0, 200.0], prior_p1=[0.5] * 4,
             step_space=[rd.RD_STEP_LOG] * 4)


def load_dataset(name):
    return np.load(os.path.join(ROOT, "data", f"{name}.npz"))


def small_dataset(n, n_steps, tau=2.5e-4, seed=0, field_mask=3, obs_frac=(1.0,), sigma=0.01):
    """A small 2-D workload built like the stored ones (steady state of the
    true parameters + seeded noise; y from the oracle + seeded noise)."""
    us, vs = oracle.steady_state(0.1, 0.9)
    noise = rd_synth.uniform_noise((2, n, n), seed, 0.01)
    u0 = (us + noise[0]).astype(np.float32).astype(np.float64)
    v0 = (vs + noise[1]).astype(np.float32).astype(np.float64)
    steps = [int(round(f * n_steps)) for f in obs_frac]
    nf = bin(field_mask).count("1")
    P = oracle.Problem(2, n, tau, n_steps, u0, v0, y=np.zeros((len(steps), nf, n, n)),
                       obs_steps=steps, field_mask=field_mask, sigma=sigma)
    _, st, _, _, clean = P.forward([0.1, 0.9, 10.0, 200.0, 0.0], want_obs=True)
    assert st == 0
    y = (clean + rd_synth.gaussian_noise(clean.shape, seed + 1, sigma)).astype(np.float32)
    return dict(u0=u0, v0=v0, y=y.astype(np.float64), obs_steps=np.array(steps), n=n,
                tau=tau, n_steps=n_steps, field_mask=field_mask, sigma=sigma)


def oracle_problem(ds, growth_r=False):
    n = ds["n"]
    return oracle.Problem(2, n, ds["tau"], ds["n_steps"], ds["u0"], ds["v0"], y=ds["y"],
                          obs_steps=ds["obs_steps"], field_mask=ds["field_mask"],
                          sigma=ds["sigma"])


def gpu_problem(datasets, solver=rd.RD_SOLVER_DCT_SIMT, growth=0, model=LOGN4, fixed=None):
    """One CUDA problem holding every dataset in `datasets` as a grid size."""
    d0 = datasets[0]
    desc = rd.make_desc(2, [d["n"] for d in datasets], d0["tau"], d0["n_steps"],
                        fixed=fixed or [0.1, 0.9, 10.0, 200.0, 0.0], solver=solver,
                        growth=growth, **model)
    p = rd.rd_problem_create(desc)
    for s, d in enumerate(datasets):
        rd.rd_set_initial_state(p, s, d["u0"], d["v0"])
        rd.rd_set_observations(p, s, d["obs_steps"], d["field_mask"], d["y"], d["sigma"])
    return p


def stored_2d(name):
    spec = rd_synth.DATASETS[name]
    ds = load_dataset(name)
    return dict(u0=ds["u0"].astype(np.float64), v0=ds["v0"].astype(np.float64),
                y=ds["y"].astype(np.float64), obs_steps=ds["obs_steps"], n=spec["n"],
                tau=spec["tau"], n_steps=spec["n_steps"], field_mask=spec["field_mask"],
                sigma=spec["sigma"])


def rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b**2).sum()))


def phi_tolerance(y, w_o, sigma, rel_field=1e-3):
    """|Phi_gpu - Phi_oracle| allowed when the fields differ by at most
    rel_field in relative L2: by Cauchy-Schwarz,
    |dPhi| <= |dw| |2 (y - w_o) - dw| / (2 sigma^2)."""
    dw = rel_field * np.sqrt((w_o**2).sum())
    r = np.sqrt(((y - w_o) ** 2).sum())
    return (dw * (2 * r + dw)) / (2 * sigma**2)
