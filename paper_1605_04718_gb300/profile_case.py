"""One batched forward solve of the stored 2-D workload, sized for profiling.

    python -m paper_1605_04718_gb300.profile_case --n 128 --proposals 152 \
        --imex-steps 400 --solver tc --launches 2

Runs `launches` rd_evaluate_batch calls (the same persistent solve kernel
the sampler uses) on `proposals` prior draws with the first `imex-steps` of
the time loop, and prints the mean kernel time from CUDA events.  The
shortened time loop keeps an ncu capture of many replay passes small.

    python -m paper_1605_04718_gb300.profile_case --mixed --proposals 4096 \
        --imex-steps 8000 --launches 2 --autotune

The uneven batch instead: the stored 64^2, 96^2 and 128^2 datasets as three
grid sizes of one problem, a third of the proposals each; with --autotune the
per-size kernel search (rd_autotune, 200-step probes) runs first and the
batch is timed with the library's default kernels and with the tuned ones.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import paper_1605_04718_gb300 as rd
    import rd_synth
    from paper_1605_04718_gb300 import build

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128, choices=[64, 96, 128])
    ap.add_argument("--proposals", type=int, default=152)
    ap.add_argument("--imex-steps", type=int, default=400)
    ap.add_argument("--solver", default="tc", choices=["tc", "simt"])
    ap.add_argument("--launches", type=int, default=2)
    ap.add_argument("--mixed", action="store_true", help="64^2, 96^2 and 128^2 in one batch")
    ap.add_argument("--autotune", action="store_true", help="with --mixed: tune kernels first")
    a = ap.parse_args()

    build.build()
    rd.load()
    if a.mixed:
        return mixed(a)
    name = f"rd2d_n{a.n}"
    spec = rd_synth.DATASETS[name]
    ds = np.load(os.path.join(ROOT, "data", f"{name}.npz"))
    steps = min(a.imex_steps, spec["n_steps"])
    solver = rd.RD_SOLVER_DCT_TC if a.solver == "tc" else rd.RD_SOLVER_DCT_SIMT
    desc = rd.make_desc(2, [a.n], spec["tau"], steps, [0, 1, 2, 3], [0.1, 0.9, 10.0, 200.0, 0.0],
                        [rd.RD_PRIOR_LOGNORMAL] * 4, [0.1, 0.9, 10.0, 200.0], [0.5] * 4,
                        [rd.RD_STEP_LOG] * 4, solver=solver)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    p = rd.rd_problem_create(desc, stream)
    rd.rd_set_initial_state(p, 0, ds["u0"].astype(np.float64), ds["v0"].astype(np.float64))
    # observe the (shortened) final step with the stored data
    rd.rd_set_observations(p, 0, [steps], spec["field_mask"], ds["y"].astype(np.float64),
                           spec["sigma"])
    theta = rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.05] * 4, a.proposals, seed=3)
    th = torch.tensor(theta, dtype=torch.float64, device=dev)
    phi = torch.zeros(a.proposals, dtype=torch.float64, device=dev)
    st = torch.zeros(a.proposals, dtype=torch.int32, device=dev)
    ms = []
    for _ in range(a.launches):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rd.rd_evaluate_batch(p, th, phi, st)
        e1.record(stream)
        rd.rd_sync(p)
        ms.append(e0.elapsed_time(e1))
    ok = int((st == 0).sum())
    per_step_proposal_us = 1e3 * np.mean(ms) / steps
    print(f"n={a.n} solver={a.solver} proposals={a.proposals} imex_steps={steps} "
          f"kernel_ms={np.mean(ms):.3f} ok={ok} us_per_step={per_step_proposal_us:.3f}")
    rd.rd_problem_destroy(p)


def _timed(rd, torch, p, stream, th, phi, st, sz, launches):
    ms = []
    for _ in range(launches):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rd.rd_evaluate_batch(p, th, phi, st, size_idx=sz)
        e1.record(stream)
        rd.rd_sync(p)
        ms.append(e0.elapsed_time(e1))
    return float(np.mean(ms))


def mixed(a):
    import json

    import torch

    import paper_1605_04718_gb300 as rd
    import rd_synth
    from paper_1605_04718_gb300.autotune import KERNEL_NAMES

    names = ["rd2d_n64", "rd2d_n96", "rd2d_n128"]
    specs = [rd_synth.DATASETS[nm] for nm in names]
    steps = min(a.imex_steps, specs[0]["n_steps"])
    desc = rd.make_desc(2, [sp["n"] for sp in specs], specs[0]["tau"], steps, [0, 1, 2, 3],
                        [0.1, 0.9, 10.0, 200.0, 0.0], [rd.RD_PRIOR_LOGNORMAL] * 4,
                        [0.1, 0.9, 10.0, 200.0], [0.5] * 4, [rd.RD_STEP_LOG] * 4,
                        solver=rd.RD_SOLVER_AUTO)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    p = rd.rd_problem_create(desc, stream)
    for s, (nm, sp) in enumerate(zip(names, specs)):
        ds = np.load(os.path.join(ROOT, "data", f"{nm}.npz"))
        rd.rd_set_initial_state(p, s, ds["u0"].astype(np.float64), ds["v0"].astype(np.float64))
        rd.rd_set_observations(p, s, [steps], sp["field_mask"], ds["y"].astype(np.float64),
                               sp["sigma"])
    B = a.proposals
    theta = rd_synth.lognormal_draws([0.1, 0.9, 10.0, 200.0], [0.05] * 4, B, seed=3)
    th = torch.tensor(theta, dtype=torch.float64, device=dev)
    sz = torch.tensor(np.arange(B) % 3, dtype=torch.int32, device=dev)
    phi = torch.zeros(B, dtype=torch.float64, device=dev)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    out = {"proposals": B, "imex_steps": steps,
           "default_kernels": [KERNEL_NAMES[rd.rd_get_size_kernel(p, s)] for s in range(3)]}
    out["default_ms"] = _timed(rd, torch, p, stream, th, phi, st, sz, a.launches)
    if a.autotune:
        times = rd.rd_autotune(p, theta[:456], n_trials=3, probe_steps=min(200, steps), n_sizes=3)
        out["autotune_us_per_proposal_step"] = {
            nm: {KERNEL_NAMES[k]: (None if not np.isfinite(t) else 1e6 * t / min(200, steps))
                 for k, t in zip((rd.RD_KERNEL_SIMT, rd.RD_KERNEL_TC_STACKED,
                                  rd.RD_KERNEL_TC_RESIDENT), times[s])}
            for s, nm in enumerate(names)}
        out["tuned_kernels"] = [KERNEL_NAMES[rd.rd_get_size_kernel(p, s)] for s in range(3)]
        out["tuned_ms"] = _timed(rd, torch, p, stream, th, phi, st, sz, a.launches)
    out["ok"] = int((st == 0).sum())
    print(json.dumps(out))
    rd.rd_problem_destroy(p)


if __name__ == "__main__":
    main()
