"""Write the synthetic observation datasets under ``data/`` (uses only the
oracle and the seeded input draws of ``rd_synth``).

Recipe per dataset (Sec. 3.1.2, "synthetic data"): the initial state is the
homogeneous steady state (a + b, b / (a + b)^2) of the true parameters plus
seeded U(-0.01, 0.01) noise per node and field, rounded to the storage type;
the oracle solves the forward problem from that state at the true parameters
in FP64; the observed fields at the observation times plus seeded
N(0, sigma^2) noise, rounded to the storage type, are the data y.  Storage is
float64 for the 1-D FP64 workload and float32 for the 2-D ones, so both sides
read bit-identical inputs.

Usage:  python -m oracle.make_datasets [name ...]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
import rd_synth  # noqa: E402

DATA_DIR = os.path.join(_ROOT, "data")


def make_example1(name):
    """Example 1 (Sec. 3.1.1): the FP64 semi-implicit solve to T = 600 under
    the true growth law, then u and v at T plus N(0, sigma^2) noise with sigma
    = 5 % of the range of u (both fields share sigma)."""
    from oracle import protocol
    spec = rd_synth.DATASETS[name]
    n = spec["n"]
    u0, v0 = protocol.example1_initial_state(n)
    P = oracle.Problem(1, n, spec["tau"], spec["n_steps"], u0, v0, scheme=spec["scheme"],
                       growth=spec["growth"], logistic_K=spec["logistic_K"])
    t0 = time.time()
    _, st, u, v = P.forward(spec["theta"])
    assert st == 0, f"{name}: true-law solve failed (status {st})"
    sigma = spec["noise_frac"] * float(u.max() - u.min())
    clean = np.stack([u, v])[None]  # [1 obs][2 fields][n]
    y = clean + rd_synth.gaussian_noise(clean.shape, spec["obs_seed"], sigma)
    path = os.path.join(DATA_DIR, f"{name}.npz")
    np.savez(path, u0=u0, v0=v0, y=y, obs_steps=np.asarray([spec["n_steps"]], np.int32),
             clean=clean, sigma=np.float64(sigma))
    print(f"{name}: {time.time() - t0:.1f} s, sigma {sigma:.4f}, u range "
          f"[{u.min():.3f}, {u.max():.3f}]")
    return path


def make(name):
    spec = rd_synth.DATASETS[name]
    if spec.get("ic") == "example1":
        return make_example1(name)
    dt = np.float64 if spec["dtype"] == "f64" else np.float32
    n, dim = spec["n"], spec["dim"]
    shape = (n,) if dim == 1 else (n, n)
    a, b = spec["theta"][0], spec["theta"][1]
    us, vs = oracle.steady_state(a, b)
    noise = rd_synth.uniform_noise((2,) + shape, spec["ic_seed"], spec["ic_amp"])
    u0 = (us + noise[0]).astype(dt)
    v0 = (vs + noise[1]).astype(dt)
    steps = rd_synth.obs_steps(spec)
    nf = bin(spec["field_mask"]).count("1")
    P = oracle.Problem(dim, n, spec["tau"], spec["n_steps"], u0.astype(np.float64),
                       v0.astype(np.float64), y=np.zeros((len(steps), nf) + shape),
                       obs_steps=steps, field_mask=spec["field_mask"], sigma=spec["sigma"])
    t0 = time.time()
    _, st, _, _, clean = P.forward(spec["theta"], want_obs=True)
    assert st == 0, f"{name}: true-parameter solve failed (status {st})"
    y = (clean + rd_synth.gaussian_noise(clean.shape, spec["obs_seed"], spec["sigma"])).astype(dt)
    os.makedirs(DATA_DIR, exist_ok=True)
    path = os.path.join(DATA_DIR, f"{name}.npz")
    np.savez(path, u0=u0, v0=v0, y=y, obs_steps=np.asarray(steps, np.int32),
             clean=clean.astype(dt))
    print(f"{name}: {time.time() - t0:.1f} s, y range [{y.min():.3f}, {y.max():.3f}]")
    return path


if __name__ == "__main__":
    names = sys.argv[1:] or list(rd_synth.DATASETS)
    for nm in names:
        make(nm)
