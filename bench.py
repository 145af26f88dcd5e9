"""Throughput benchmark: batched random-walk Metropolis on the 128^2
Schnakenberg workload (forward solves/s), through the library's C ABI.

One "step" = one MCMC step of every chain: propose, 8000-step IMEX forward
solve + Gaussian log-likelihood of every proposal, accept/reject (Algorithm 1).
value = exact forward solves per second over all GPUs (weak scaling: each rank
runs its own chains, no collective on the data path).

On one GPU the line also carries, each measured in the same run:
  workloads  the other batched workloads -- 64^2 plain chains (1024 chains),
             the uneven 64^2/96^2/128^2 batch (4096 proposals per launch,
             autotuned kernels) and the growing 128^2 domain (50000 steps,
             2048 chains, five parameters) -- each with its HBM-normalised
             fraction;
  ess        plain against delayed-acceptance sampling: ESS/s at the same
             posterior, chains run until split-R-hat < 1.01, posterior
             agreement in Monte Carlo standard errors.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rd_synth  # noqa: E402

DATASET = "rd2d_n128"
TRUE4 = [0.1, 0.9, 10.0, 200.0]
METRIC = "forward solves/s (128^2, 8000 IMEX steps/solve)"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# RD_KERNEL_* of include/rdbayes.h
KERNELS = {"simt": 1, "stacked": 2, "resident": 3}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per full launch
# (4096 proposals x 8000 steps at 128^2) of a solve kernel, from an ncu capture;
# reported only while the SHA-256 of the kernel's sources still matches the
# one the capture ran on, else null.
TRAFFIC = {
    "k_solve2d_tc128<2>": {
        "sha256": "a6fb8214b6386bfa77af795dbeec585ed5d7c2da3421f652fea7b86df8117e2c",
        "bytes": 1102336 + 256,
    },
}
TRAFFIC_SOURCES = {  # the kernel's own code (its loads and stores)
    "k_solve2d_tc128<2>": ["rd_solve_tc2.cu", "rd_tc_ptx.cuh"],
}


def sources_sha256(kernel):
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_1605_04718_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_of(kernel):
    t = TRAFFIC.get(kernel)
    if t and kernel in TRAFFIC_SOURCES and t["sha256"] == sources_sha256(kernel):
        return t["bytes"]
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def _find(d, *keys):
    for k in keys:
        if isinstance(d, dict) and k in d and isinstance(d[k], (int, float)):
            return float(d[k])
    if isinstance(d, dict):
        for v in d.values():
            r = _find(v, *keys) if isinstance(v, dict) else None
            if r is not None:
                return r
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to RD_CLOCKS_DIR (if set) or the system temp directory
        out_dir = os.environ.get("RD_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_gpu{gpu_index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_config(chains):
    spec = rd_synth.DATASETS[DATASET]
    return {"workload": f"batched plain RW-Metropolis, Schnakenberg 2-D {spec['n']}^2, "
                        f"tau={spec['tau']}, {spec['n_steps']} IMEX steps/solve (T=2), "
                        f"4 params (a,b,d,gamma) log-normal priors, {chains} chains x 1 proposal/step",
            "grid": spec["n"], "imex_steps": spec["n_steps"], "chains": chains,
            "l2": "L2 (129 MB) flushed with a 512 MB write between timed steps"}


def cpu_baseline(sample_steps=None, cores=None):
    """Oracle forward solves on the host cores (one proposal per thread) over a
    bounded number of IMEX steps, scaled to full 8000-step solves."""
    import oracle
    oracle.build()
    spec = rd_synth.DATASETS[DATASET]
    ds = np.load(os.path.join(ROOT, "data", f"{DATASET}.npz"))
    cores = cores or os.cpu_count() or 1
    sample_steps = sample_steps or 600
    P = oracle.Problem(2, spec["n"], spec["tau"], sample_steps, ds["u0"].astype(np.float64),
                       ds["v0"].astype(np.float64), y=ds["y"].astype(np.float64),
                       obs_steps=[sample_steps], field_mask=3, sigma=spec["sigma"])
    theta = rd_synth.lognormal_draws(TRUE4, [0.05] * 4, cores, seed=1)
    theta = np.concatenate([theta, np.zeros((cores, 1))], 1)
    t0 = time.perf_counter()
    P.forward_batch(theta, n_threads=cores)
    dt = time.perf_counter() - t0
    solves = cores * sample_steps / spec["n_steps"]
    return {"value": solves / dt, "unit": "forward solves/s", "cores": cores, "kind": "oracle",
            "wall_s": dt,
            "sample": f"{cores} proposals x {sample_steps} of {spec['n_steps']} IMEX steps "
                      f"at {spec['n']}^2 (FP64, one proposal per host thread), scaled to full "
                      f"solves; {dt:.1f} s wall"}


def run_reference(args):
    """The oracle timed as it stands: each step solves one proposal per host
    core for ref_sample_steps of the 8000 IMEX steps; ms_per_step is that
    step's measured wall time and value the rate scaled to full solves."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    runs = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(sample_steps=args.ref_sample_steps)
        if i >= args.warmup:
            runs.append(r)
    value = float(np.mean([r["value"] for r in runs]))
    spec = rd_synth.DATASETS[DATASET]
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "forward solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean([r["wall_s"] for r in runs])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.chains),
            "scaled": {"step": f"{runs[-1]['cores']} proposals x {args.ref_sample_steps} of "
                               f"{spec['n_steps']} IMEX steps (one per host thread)",
                       "value": "solves/s scaled to full 8000-step solves",
                       "full_4096_chain_step_s_extrapolated": args.chains / value},
            "cpu_baseline": {"value": value, "unit": "forward solves/s",
                             "cores": runs[-1]["cores"], "kind": "oracle",
                             "sample": runs[-1]["sample"]},
            "e2e": {"value": value, "unit": "forward solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------- helpers
def make_problem(rd, names, stream, growth=False, kernel=None, steps=None):
    """A problem over the stored datasets `names` (one grid size each)."""
    specs = [rd_synth.DATASETS[nm] for nm in names]
    sp0 = specs[0]
    n_steps = steps or sp0["n_steps"]
    if growth:
        desc = rd.make_desc(2, [s["n"] for s in specs], sp0["tau"], n_steps, [0, 1, 2, 3, 4],
                            list(sp0["theta"]),
                            [rd.RD_PRIOR_LOGNORMAL] * 4 + [rd.RD_PRIOR_UNIFORM],
                            TRUE4 + [0.0], [0.5] * 4 + [0.05],
                            [rd.RD_STEP_LOG] * 4 + [rd.RD_STEP_LINEAR], growth=1)
    else:
        desc = rd.make_desc(2, [s["n"] for s in specs], sp0["tau"], n_steps, [0, 1, 2, 3],
                            [0.1, 0.9, 10.0, 200.0, 0.0], [rd.RD_PRIOR_LOGNORMAL] * 4, TRUE4,
                            [0.5] * 4, [rd.RD_STEP_LOG] * 4)
    p = rd.rd_problem_create(desc, stream)
    for s, (nm, sp) in enumerate(zip(names, specs)):
        ds = np.load(os.path.join(ROOT, "data", f"{nm}.npz"))
        rd.rd_set_initial_state(p, s, ds["u0"].astype(np.float64), ds["v0"].astype(np.float64))
        y = ds["y"].astype(np.float64)
        obs = ds["obs_steps"]
        if steps is not None:  # a shortened run observes its last step against the last data
            obs, y = [n_steps], y[-1:]
        rd.rd_set_observations(p, s, obs, sp["field_mask"], y, sp["sigma"])
        if kernel is not None:
            rd.rd_set_size_kernel(p, s, kernel)
    return p


def timed(torch, stream, fn, reps, flush=None):
    """Seconds of each of `reps` calls of fn, CUDA events on `stream`, the L2
    flushed before each."""
    out = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(3.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1) / 1e3)
    return out


def hbm_equiv(n, steps, solves_per_s, hbm):
    gbs = 16.0 * n * n * steps * solves_per_s / 1e9
    return {"gbs": gbs, "frac": gbs / hbm}


def chain_workload(rd, torch, stream, dev, flush, name, C, step, growth, warmup, reps, hbm):
    spec = rd_synth.DATASETS[name]
    p = make_problem(rd, [name], stream, growth=growth)
    centre = list(spec["theta"]) if growth else TRUE4
    theta0 = rd_synth.chain_starts(centre, C, seed=2000 + spec["n"], rel=0.002)
    c = rd.rd_chains_create(p, theta0, 4343, step, capacity=warmup + reps + 1)
    for _ in range(warmup):
        rd.rd_chains_run(c, 1)
    torch.cuda.synchronize(dev)
    t = timed(torch, stream, lambda: rd.rd_chains_run(c, 1), reps, flush)
    _, cnt = rd.rd_chains_read_samples(c, warmup + reps + 1, len(step), C)
    solves_per_step = cnt[3] / cnt[0] * C
    value = solves_per_step / float(np.mean(t))
    out = {"workload": f"plain chains, {spec['n']}^2, {spec['n_steps']} IMEX steps/solve, "
                       f"{C} chains, {len(step)} params" + (", growing domain" if growth else ""),
           "value": value, "unit": "forward solves/s", "ms_per_step": 1e3 * float(np.mean(t)),
           "steps": reps, "warmup": warmup,
           "kernel": {1: "simt", 2: "tc_stacked", 3: "tc_resident",
                      4: "cg"}[rd.rd_get_size_kernel(p, 0)],
           "hbm_equiv": hbm_equiv(spec["n"], spec["n_steps"], value, hbm),
           "accept_rate": float(cnt[2] / max(cnt[0], 1))}
    rd.rd_chains_destroy(c)
    rd.rd_problem_destroy(p)
    return out


def mixed_workload(rd, torch, stream, dev, flush, hbm, B=4096, launches=3):
    """The uneven batch: 64^2, 96^2 and 128^2 (a third each) in one
    evaluation, kernels per size chosen by the timed search."""
    from paper_1605_04718_gb300.autotune import KERNEL_NAMES
    names = ["rd2d_n64", "rd2d_n96", "rd2d_n128"]
    ns = [rd_synth.DATASETS[nm]["n"] for nm in names]
    steps = rd_synth.DATASETS[names[0]]["n_steps"]
    p = make_problem(rd, names, stream)
    theta = rd_synth.lognormal_draws(TRUE4, [0.002] * 4, B, seed=3)
    t0 = time.perf_counter()
    tune = rd.rd_autotune(p, theta[:456], n_trials=3, probe_steps=200, n_sizes=3)
    t_tune = time.perf_counter() - t0
    kinds = [rd.rd_get_size_kernel(p, s) for s in range(3)]
    th = torch.tensor(theta, dtype=torch.float64, device=dev)
    sz_np = (np.arange(B) % 3).astype(np.int32)
    sz = torch.tensor(sz_np, device=dev)
    phi = torch.zeros(B, dtype=torch.float64, device=dev)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    rd.rd_evaluate_batch(p, th, phi, st, size_idx=sz)
    rd.rd_sync(p)
    t = timed(torch, stream, lambda: rd.rd_evaluate_batch(p, th, phi, st, size_idx=sz),
              launches, flush)
    rd.rd_sync(p)
    ok = int((st == 0).sum())
    t_mix = float(np.mean(t))
    # each kernel kind's launch alone (its sizes' proposals only)
    per_kind = {}
    for kind in sorted(set(kinds)):
        sel = np.nonzero(np.isin(sz_np, [s for s in range(3) if kinds[s] == kind]))[0]
        th_k = th[torch.tensor(sel, device=dev)].contiguous()
        sz_k = sz[torch.tensor(sel, device=dev)].contiguous()
        ph_k = torch.zeros(len(sel), dtype=torch.float64, device=dev)
        st_k = torch.zeros(len(sel), dtype=torch.int32, device=dev)
        tk = timed(torch, stream, lambda: rd.rd_evaluate_batch(p, th_k, ph_k, st_k, size_idx=sz_k),
                   2, flush)
        per_kind[KERNEL_NAMES[kind]] = {"proposals": int(len(sel)), "ms": 1e3 * float(np.mean(tk))}
    rd.rd_sync(p)
    rd.rd_problem_destroy(p)
    value = B / t_mix
    bytes_per_s = sum(16.0 * n * n * steps * (B / 3) for n in ns) / t_mix
    return {"workload": f"uneven batch 64^2/96^2/128^2 (1/3 each), {steps} IMEX steps/solve, "
                        f"{B} proposals per evaluation",
            "value": value, "unit": "forward solves/s", "ms_per_launch_set": 1e3 * t_mix,
            "launches": launches, "ok": ok,
            "kernels": {str(n): KERNEL_NAMES[k] for n, k in zip(ns, kinds)},
            "autotune_us_per_proposal_step": {
                str(n): {KERNEL_NAMES[k]: (None if not np.isfinite(x) else 1e6 * x / 200)
                         for k, x in zip((1, 2, 3, 4), tune[s])} for s, n in enumerate(ns)},
            "autotune_s": t_tune,
            "per_kernel_launch": per_kind,
            "hbm_equiv": {"gbs": bytes_per_s / 1e9, "frac": bytes_per_s / 1e9 / hbm}}


# ----------------------------------------------------------------- ESS/s
def _agreement(sa, sb):
    """Largest |difference| / combined MCSE over parameters of the posterior
    mean and the 2.5% / 97.5% quantiles of two summaries."""
    z = []
    for a, b in zip(sa, sb):
        z.append(abs(a["mean"] - b["mean"]) / np.hypot(a["mcse"], b["mcse"]))
        z.append(abs(a["q025"] - b["q025"]) / np.hypot(a["mcse_q025"], b["mcse_q025"]))
        z.append(abs(a["q975"] - b["q975"]) / np.hypot(a["mcse_q975"], b["mcse_q975"]))
    return float(max(z))


def ess_comparison(rd, torch, p, stream, dev, C_full, plain_step_s, args):
    """ESS per second of plain and delayed-acceptance sampling on the bench
    workload.  ESS per chain-step comes from 152-chain runs (one chain per SM)
    of both samplers from the same tuned starts, extended in blocks until
    split-R-hat < 1.01 for every parameter of both (first quarter discarded);
    the cost of a chain-step comes from timed steps of C_full chains."""
    from paper_1605_04718_gb300 import stats
    names = ["a", "b", "d", "gamma"]
    t_total0 = time.perf_counter()
    Cp = 152
    # pilot: start near the mode, adapt the log-space steps towards an
    # acceptance rate of 0.2-0.35, then a proposal covariance from the spread
    theta = np.asarray(rd_synth.chain_starts(TRUE4, Cp, seed=7000, rel=2e-4))
    step = np.array([1e-4, 1e-4, 1e-4, 1e-4])
    L = np.diag(step)
    scale = 1.0
    pilot = []
    for rnd in range(10):
        c = rd.rd_chains_create(p, theta, 9000 + rnd, step, capacity=25)
        rd.rd_chains_set_proposal(c, scale * L)
        rd.rd_chains_run(c, 25)
        smp, cnt = rd.rd_chains_read_samples(c, 25, 4, Cp)
        theta, _ = rd.rd_chains_get_state(c, 4, Cp)
        rd.rd_chains_destroy(c)
        acc = cnt[2] / max(cnt[0], 1)
        pilot.append((acc, np.log(smp)))
        scale *= 0.4 if acc < 0.05 else 0.7 if acc < 0.15 else 1.4 if acc > 0.4 else 1.0
        if rnd >= 3:  # covariance of log theta from the last rounds, within-chain centred
            lsm = np.concatenate([x[1] for x in pilot[-4:]], 0)
            dev_ = (lsm - lsm.mean(0, keepdims=True)).transpose(1, 0, 2).reshape(4, -1)
            cov = np.cov(dev_) + 1e-18 * np.eye(4)
            L = np.linalg.cholesky(2.38 ** 2 / 4 * cov)
            if rnd == 3:
                scale = 1.0
    lt = np.concatenate([x[1] for x in pilot[-4:]], 0).transpose(1, 0, 2).reshape(4, -1)
    mu = lt.mean(1)
    cov = np.cov(lt) + 1e-18 * np.eye(4)
    Lc = np.linalg.cholesky(cov)
    prop = scale * L
    # training pairs from the batched exact solver
    t0 = time.perf_counter()
    rng = np.random.default_rng(11)
    if args.ess_train == "prior":  # draws from the log-normal prior itself
        n_train = args.ess_train_pairs or 200000
        th_tr = rd_synth.lognormal_draws(TRUE4, [0.5] * 4, n_train, seed=7)
    else:  # around the pilot's posterior, 2.5 posterior sd wide
        n_train = args.ess_train_pairs or 8192
        th_tr = np.exp(mu[None, :] + 2.5 * rng.standard_normal((n_train, 4)) @ Lc.T)
    th_d = torch.tensor(th_tr, dtype=torch.float64, device=dev)
    phi_d = torch.zeros(n_train, dtype=torch.float64, device=dev)
    st_d = torch.zeros(n_train, dtype=torch.int32, device=dev)
    for i in range(0, n_train, 16384):
        j = min(n_train, i + 16384)
        rd.rd_evaluate_batch(p, th_d[i:j], phi_d[i:j], st_d[i:j])
    rd.rd_sync(p)
    t_gen = time.perf_counter() - t0
    n_ok = int((st_d == 0).sum())
    t0 = time.perf_counter()
    sur = rd.rd_surrogate_create(p, seed=5)
    rep = rd.rd_surrogate_train(sur, th_d, phi_d, epochs=args.ess_epochs, batch=1024, lr=1e-3,
                                holdout_frac=0.1, seed=3)
    t_train = time.perf_counter() - t0
    # the surrogate's error on the posterior itself (pilot draws, exact Phi)
    th_post = np.exp(mu[None, :] + rng.standard_normal((1024, 4)) @ Lc.T)
    thp = torch.tensor(th_post, dtype=torch.float64, device=dev)
    ph_ex = torch.zeros(1024, dtype=torch.float64, device=dev)
    st_ex = torch.zeros(1024, dtype=torch.int32, device=dev)
    ph_su = torch.zeros(1024, dtype=torch.float64, device=dev)
    rd.rd_evaluate_batch(p, thp, ph_ex, st_ex)
    rd.rd_surrogate_predict(sur, thp, ph_su)
    rd.rd_sync(p)
    e_post = (ph_su - ph_ex).cpu().numpy()
    out = {"proposal_chol_log": prop.tolist(), "pilot_accept": [x[0] for x in pilot],
           "posterior_sd_log": np.sqrt(np.diag(cov)).tolist(),
           "train": args.ess_train, "train_pairs": n_train, "train_pairs_ok": n_ok,
           "surrogate_holdout_rel_err": float(rep[2]),
           "surrogate_posterior_err_sd": float(e_post.std()),
           "t_datagen_s": t_gen, "t_train_s": t_train}
    # both samplers from the same starts, in blocks until split-R-hat < 1.01
    chains = {}
    for mode in ("plain", "da"):
        c = rd.rd_chains_create(p, theta, 424242, step, capacity=args.ess_block)
        rd.rd_chains_set_proposal(c, prop)
        if mode == "da":
            rd.rd_chains_set_surrogate(c, sur)
        chains[mode] = [c, [], None]
    done, total = False, 0
    while not done and total < args.ess_max_steps:
        for mode in ("plain", "da"):
            rd.rd_chains_run(chains[mode][0], args.ess_block)
        for mode in ("plain", "da"):
            smp, cnt = rd.rd_chains_read_samples(chains[mode][0], args.ess_block, 4, Cp)
            chains[mode][1].append(smp)
            chains[mode][2] = cnt
        total += args.ess_block
        done = all(max(x["rhat"] for x in stats.summarize(np.concatenate(chains[m][1], 0),
                                                          burn_frac=0.25, names=names)) < 1.01
                   for m in ("plain", "da"))
    res, summ = {}, {}
    for mode in ("plain", "da"):
        smp = np.concatenate(chains[mode][1], 0)
        cnt = chains[mode][2]
        rd.rd_chains_destroy(chains[mode][0])
        sm = stats.summarize(smp, burn_frac=0.25, names=names)
        summ[mode] = sm
        kept = smp.shape[0] - int(np.floor(0.25 * smp.shape[0]))
        ess_min = min(x["ess"] for x in sm)
        res[mode] = {"ess_per_chain_step": ess_min / (kept * Cp), "ess_min": ess_min,
                     "steps": int(smp.shape[0]), "accept": cnt[2] / cnt[0],
                     "solves_per_step": cnt[3] / cnt[0],
                     "mean": [x["mean"] for x in sm], "q025": [x["q025"] for x in sm],
                     "q975": [x["q975"] for x in sm],
                     "rhat_max": max(x["rhat"] for x in sm)}
    # cost of a full-batch delayed-acceptance step (C_full chains)
    th_full = np.exp(mu[None, :] + np.random.default_rng(5).standard_normal((C_full, 4)) @ Lc.T)
    c = rd.rd_chains_create(p, th_full, 777, step, capacity=8)
    rd.rd_chains_set_proposal(c, prop)
    rd.rd_chains_set_surrogate(c, sur)
    rd.rd_chains_run(c, 2)
    rd.rd_sync(p)
    da_step_s = float(np.mean(timed(torch, stream, lambda: rd.rd_chains_run(c, 1), 4)))
    rd.rd_chains_destroy(c)
    rd.rd_surrogate_destroy(sur)
    plain_ess_s = res["plain"]["ess_per_chain_step"] * C_full / plain_step_s
    da_ess_s = res["da"]["ess_per_chain_step"] * C_full / da_step_s
    run_steps = 5000
    da_total = t_gen + t_train + run_steps * da_step_s
    z = _agreement(summ["da"], summ["plain"])
    out.update({
        "plain": res["plain"], "da": res["da"],
        "rhat_below_1.01": bool(done),
        "posterior_agreement": {"max_z": z, "within_3_mcse": z < 3.0,
                                "what": "max over (a,b,d,gamma) of |DA - plain| / combined MCSE "
                                        "of the mean and of the 2.5%/97.5% quantiles"},
        "plain_step_s_at_full_batch": plain_step_s, "da_step_s_at_full_batch": da_step_s,
        "ess_per_s_plain": plain_ess_s, "ess_per_s_da": da_ess_s,
        "ess_per_s_da_amortised_projected_5000_steps":
            res["da"]["ess_per_chain_step"] * C_full * run_steps / da_total,
        "exact_solves_per_ess": {
            m: res[m]["solves_per_step"] / res[m]["ess_per_chain_step"] for m in ("plain", "da")},
        "da_vs_plain": da_ess_s / plain_ess_s,
        "method": f"ESS = min over (a,b,d,gamma) of the multi-chain ESS of {Cp} chains run in "
                  f"blocks of {args.ess_block} steps until split-R-hat < 1.01 (cap "
                  f"{args.ess_max_steps}), first quarter discarded, from a pilot with an adapted "
                  f"proposal covariance (Haario et al. 2001); cost per step from {C_full}-chain "
                  "steps; the amortised figure adds the measured data-generation and training "
                  "time to a projected 5000-step run",
        "t_wall_s": time.perf_counter() - t_total0,
    })
    return out


def run_case(args):
    """One stored 2-D workload, solves only, sized for profiling: `launches`
    rd_evaluate_batch calls over `proposals` draws near the true parameters
    with the first `steps` IMEX steps of the time loop; prints the mean
    launch time (CUDA events) as one JSON line."""
    import torch

    import paper_1605_04718_gb300 as rd
    from paper_1605_04718_gb300 import build as rdbuild
    rdbuild.build()
    rd.load()
    name = f"rd2d_n{args.case_n}"
    spec = rd_synth.DATASETS[name]
    steps = min(args.case_steps, spec["n_steps"])
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    p = make_problem(rd, [name], stream, steps=steps,
                     kernel=None if args.kernel == "default" else KERNELS[args.kernel])
    if args.case_ctas:
        rd.rd_set_size_schedule(p, 0, args.case_ctas)
    B = args.case_proposals
    theta = rd_synth.lognormal_draws(TRUE4, [0.05] * 4, B, seed=3)
    th = torch.tensor(theta, dtype=torch.float64, device=dev)
    phi = torch.zeros(B, dtype=torch.float64, device=dev)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    t = timed(torch, stream, lambda: rd.rd_evaluate_batch(p, th, phi, st), args.case_launches)
    rd.rd_sync(p)
    kind = {1: "simt", 2: "tc_stacked", 3: "tc_resident", 4: "cg"}[rd.rd_get_size_kernel(p, 0)]
    print(json.dumps({"case": name, "proposals": B, "imex_steps": steps, "kernel": kind,
                      "ctas_per_sm": rd.rd_get_size_schedule(p, 0),
                      "launch_ms": 1e3 * float(np.mean(t)), "ok": int((st == 0).sum()),
                      "us_per_proposal_step": 1e6 * float(np.mean(t)) / (B * steps),
                      "solves_per_s_at_8000_steps": B / (float(np.mean(t)) * 8000 / steps)}))
    rd.rd_problem_destroy(p)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1605_04718_gb300 as rd
    from paper_1605_04718_gb300 import build as rdbuild
    from paper_1605_04718_gb300 import shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        rdbuild.build()
    if world > 1:
        dist.barrier()
    rd.load()

    spec = rd_synth.DATASETS[DATASET]
    n, C = spec["n"], args.chains
    stream = torch.cuda.current_stream(dev)
    p = make_problem(rd, [DATASET], stream,
                     kernel=None if args.kernel == "default" else KERNELS[args.kernel])
    # weak scaling: C chains per GPU, rank r runs chains [r C, (r + 1) C) of one
    # run of C * world chains (same seed, global chain index in the counters)
    first, count = shard.shard(C * world, world, rank)
    theta0 = rd_synth.chain_starts(TRUE4, C * world, seed=1000, rel=0.002)[first:first + count]
    step = [2e-4, 2e-4, 5e-4, 5e-4]
    cap = args.warmup + args.steps + 1
    chains = rd.rd_chains_create(p, theta0, 4242, step, capacity=cap)
    rd.rd_chains_set_first_chain(chains, first)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        rd.rd_chains_run(chains, 1)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    times = timed(torch, stream, lambda: rd.rd_chains_run(chains, 1), args.steps, flush)
    barrier()
    ck = clocks.stop()
    t_rank = float(np.sum(times))
    samples, counters = rd.rd_chains_read_samples(chains, cap, 4, C)
    solves_rank = float(counters[3]) * args.steps / (args.warmup + args.steps)
    # cross-check: the batch evaluation alone (work-list fill + solve), same
    # launch configuration, on the chains' states
    th = torch.tensor(samples[-1].T.copy(), dtype=torch.float64, device=dev)
    phi_d = torch.zeros(C, dtype=torch.float64, device=dev)
    st_d = torch.zeros(C, dtype=torch.int32, device=dev)
    kt = timed(torch, stream, lambda: rd.rd_evaluate_batch(p, th, phi_d, st_d),
               max(1, args.kernel_reps), flush)
    k_standalone = float(np.mean(kt))
    # end to end: host theta (pinned) in, host Phi/status out, through the C ABI
    th_h = torch.tensor(samples[-1].T.copy(), dtype=torch.float64).pin_memory().numpy()
    e2e_t = []
    for _ in range(max(1, args.e2e_reps)):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rd.rd_evaluate_batch_host(p, th_h)
        e2e_t.append(time.perf_counter() - t0)
    e2e_rank = C / float(np.mean(e2e_t))

    if world > 1:
        tt = torch.tensor([t_rank, solves_rank, e2e_rank], dtype=torch.float64, device=dev)
        tmax = tt.clone()
        dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        tsum = tt.clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        t_all, solves_all, e2e_all = float(tmax[0]), float(tsum[1]), float(tsum[2])
    else:
        t_all, solves_all, e2e_all = t_rank, solves_rank, e2e_rank

    if rank == 0:
        pk, pk_src = peaks()
        value = solves_all / t_all
        flop_per_solve = 16.0 * n**3 * spec["n_steps"]  # 4 transforms x 2 N^3 x 2 fields / step
        bytes_per_solve = 16.0 * n * n * spec["n_steps"]  # u, v FP32 read + write per step
        kind = rd.rd_get_size_kernel(p, 0)
        # the solve kernel's launch duration, taken from the timed steps: one
        # launch per step, 99.997 % of the step's device time (the ncu launch
        # list), so achieved figures are lower bounds
        k_dur = t_all / args.steps
        achieved = flop_per_solve * C / k_dur / 1e12
        if kind == rd.RD_KERNEL_SIMT:
            fp32_peak = 152 * 128 * 2 * (ck.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp32_peak, "traffic": None,
                    "kernel": "k_solve2d_simt<128,1>",
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
        else:
            tpk = _find(pk, "bf16_tflops_sustained") or FALLBACK_PEAKS["bf16_tflops_sustained"]
            kname = ("k_solve2d_tc128<2>" if kind == rd.RD_KERNEL_TC_RESIDENT
                     else "k_solve2d_tc<128>")
            roof = {"bound": "tensor", "achieved": achieved, "peak": tpk, "unit": "TFLOP/s",
                    "frac": achieved / tpk, "traffic": traffic_of(kname), "kernel": kname,
                    "peak_source": f"{pk_src} bf16 sustained (= fp16 rate): the kernel runs "
                                   "seconds at a time inside a long step"}
        roof.update({"kernel_ms": 1e3 * k_dur,
                     "kernel_ms_from": "the timed MCMC steps (one solve launch per step; the "
                                       "other kernels of a step take 0.003 % of it)",
                     "standalone_ms": 1e3 * k_standalone, "standalone_reps": len(kt),
                     "standalone_ms_each": [1e3 * x for x in kt],
                     "work": "16 N^3 flop per proposal-step (4 transforms x 2 N^3 x 2 fields) "
                             f"x {spec['n_steps']} steps x {C} proposals per launch"})
        hbm = _find(pk, "hbm_gbs", "hbm_GBps", "copy_gbs") or FALLBACK_PEAKS["hbm_gbs"]
        roof["hbm_equiv"] = {"gbs": bytes_per_solve * C / k_dur / 1e9, "peak_gbs": hbm,
                             "frac": bytes_per_solve * C / k_dur / 1e9 / hbm,
                             "note": "16 N^2 B per proposal-step; state is resident in shared "
                                     "and tensor memory, so this is the HBM-normalised rate, "
                                     "not traffic"}
        line = {
            "metric": METRIC,
            "value": value, "unit": "forward solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(C),
            "roofline": roof,
            "e2e": {"value": e2e_all, "unit": "forward solves/s",
                    "h2d_bytes_per_step": int(C * 4 * 8), "d2h_bytes_per_step": int(C * 12),
                    "call": "rd_evaluate_batch_host (pinned host theta in, host Phi/status "
                            "out, copies inside the timed call)"},
            "gpu_launches": 4 * args.steps,
            "clocks": ck,
            "accept_rate": float(counters[2] / max(counters[0], 1)),
            "peaks_source": pk_src,
        }
    rd.rd_chains_destroy(chains)
    if rank == 0 and world == 1:
        if not args.no_workloads:
            w = {}
            w["chains_64sq_1024"] = chain_workload(rd, torch, stream, dev, flush, "rd2d_n64", 1024,
                                                   [4e-4, 4e-4, 1e-3, 1e-3], False, 2, 5, hbm)
            w["uneven_64_96_128_4096"] = mixed_workload(rd, torch, stream, dev, flush, hbm)
            w["grow128_50000_2048"] = chain_workload(rd, torch, stream, dev, flush,
                                                     "rd2d_n128_grow", 2048,
                                                     [2e-4, 2e-4, 5e-4, 5e-4, 1e-5], True, 1, 2,
                                                     hbm)
            line["workloads"] = w
        if not args.no_ess:
            line["ess"] = ess_comparison(rd, torch, p, stream, dev, C, t_all / args.steps, args)
            line["ess_per_s"] = {"plain": line["ess"]["ess_per_s_plain"],
                                 "da_surrogate": line["ess"]["ess_per_s_da"]}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    rd.rd_problem_destroy(p)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--chains", type=int, default=4096)
    ap.add_argument("--kernel", default="default", choices=["default"] + sorted(KERNELS),
                    help="solve kernel of the 128^2 size (default: the library's choice)")
    ap.add_argument("--kernel-reps", type=int, default=5)
    ap.add_argument("--e2e-reps", type=int, default=1)
    ap.add_argument("--ref-sample-steps", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-ess", action="store_true", help="skip the ESS/s comparison")
    ap.add_argument("--ess-train", default="near", choices=["near", "prior"],
                    help="surrogate training pairs: around the pilot posterior or prior draws")
    ap.add_argument("--ess-train-pairs", type=int, default=0)
    ap.add_argument("--ess-epochs", type=int, default=60)
    ap.add_argument("--ess-block", type=int, default=200)
    ap.add_argument("--ess-max-steps", type=int, default=3000)
    ap.add_argument("--case-n", type=int, default=0,
                    help="solves only: stored 2-D workload of this grid (64, 96, 128)")
    ap.add_argument("--case-proposals", type=int, default=152)
    ap.add_argument("--case-steps", type=int, default=8000)
    ap.add_argument("--case-launches", type=int, default=2)
    ap.add_argument("--case-ctas", type=int, default=0, help="CTAs per SM (0: default)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.case_n:
        run_case(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
