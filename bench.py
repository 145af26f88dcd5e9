"""Throughput benchmark: batched random-walk Metropolis on the 128^2
Schnakenberg workload (forward solves/s), through the library's C ABI.

One "step" = one MCMC step of every chain: propose, 8000-step IMEX forward
solve + Gaussian log-likelihood of every proposal, accept/reject (Algorithm 1).
value = exact forward solves per second over all GPUs (weak scaling: each rank
runs its own chains, no collective on the data path).

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
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# RD_KERNEL_* of include/rdbayes.h
KERNELS = {"simt": 1, "stacked": 2, "resident": 3}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one full launch
# (4096 proposals x 8000 steps at 128^2) of a solve kernel, from one ncu
# capture of that launch (profiles/); reported only while the SHA-256 of the
# kernel's sources still matches the one the capture ran on, else null.
TRAFFIC = {
    "k_solve2d_tc128<2>": {
        "sha256": "321b2b19b49a1dbfc5af33660910825eb08659c07718ee4bc72d28acdd46b6da",
        "bytes": 1243392 + 0,  # profiles/k_solve2d_tc128_128sq_traffic.md
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
            "sample": f"{cores} proposals x {sample_steps} of {spec['n_steps']} IMEX steps "
                      f"at {spec['n']}^2 (FP64, one proposal per host thread), scaled to full "
                      f"solves; {dt:.1f} s wall"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(sample_steps=args.ref_sample_steps)
        if i >= args.warmup:
            steps.append(r)
    value = float(np.mean([r["value"] for r in steps]))
    spec = rd_synth.DATASETS[DATASET]
    line = {"impl": "reference", "metric": "forward solves/s (128^2, 8000 IMEX steps/solve)",
            "value": value, "unit": "forward solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * args.chains / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.chains),
            "cpu_baseline": {"value": value, "unit": "forward solves/s",
                             "cores": steps[-1]["cores"], "kind": "oracle",
                             "sample": steps[-1]["sample"]},
            "e2e": {"value": value, "unit": "forward solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def ess_comparison(rd, torch, p, stream, dev, C_full, plain_step_s, steps=200, seed=0):
    """ESS per second of plain and delayed-acceptance sampling on the bench
    workload.  ESS per chain-step comes from 152-chain runs (one chain per SM)
    started from a tuned pilot; the cost of a chain-step comes from timed
    steps of C_full chains.  Returns a dict for the JSON line."""
    from paper_1605_04718_gb300 import stats
    t_total0 = time.perf_counter()
    Cp = 152
    # pilot: start near the mode, adapt the log-space steps towards an
    # acceptance rate of 0.2-0.35 (per-parameter scales from the within-chain
    # spread once chains move)
    theta = np.asarray(rd_synth.chain_starts(TRUE4, Cp, seed=7000 + seed, rel=2e-4))
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
    sdv = np.sqrt(np.diag(cov))
    prop = scale * L
    # training pairs from the batched exact solver around the pilot posterior
    t0 = time.perf_counter()
    n_train = 8192
    rng = np.random.default_rng(11 + seed)
    th_tr = np.exp(mu[None, :] + 2.5 * rng.standard_normal((n_train, 4)) @ Lc.T)
    th_d = torch.tensor(th_tr, dtype=torch.float64, device=dev)
    phi_d = torch.zeros(n_train, dtype=torch.float64, device=dev)
    st_d = torch.zeros(n_train, dtype=torch.int32, device=dev)
    rd.rd_evaluate_batch(p, th_d, phi_d, st_d)
    rd.rd_sync(p)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    sur = rd.rd_surrogate_create(p, seed=5)
    rep = rd.rd_surrogate_train(sur, th_d, phi_d, epochs=60, batch=1024, lr=1e-3,
                                holdout_frac=0.1, seed=3)
    t_train = time.perf_counter() - t0
    out = {"proposal_chol_log": prop.tolist(), "pilot_accept": [x[0] for x in pilot],
           "posterior_sd_log": sdv.tolist(), "train_pairs": n_train,
           "surrogate_holdout_rel_err": float(rep[2]), "t_datagen_s": t_gen,
           "t_train_s": t_train}
    # ESS per chain-step, plain and delayed acceptance, same starts
    res = {}
    for mode in ("plain", "da"):
        c = rd.rd_chains_create(p, theta, 424242, step, capacity=steps)
        rd.rd_chains_set_proposal(c, prop)
        if mode == "da":
            rd.rd_chains_set_surrogate(c, sur)
        rd.rd_chains_run(c, steps)
        smp, cnt = rd.rd_chains_read_samples(c, steps, 4, Cp)
        rd.rd_chains_destroy(c)
        summ = stats.summarize(smp, burn_frac=0.0, names=["a", "b", "d", "gamma"])
        ess_min = min(x["ess"] for x in summ)
        res[mode] = {"ess_per_chain_step": ess_min / (steps * Cp),
                     "accept": cnt[2] / cnt[0], "solves_per_step": cnt[3] / cnt[0],
                     "mean": [x["mean"] for x in summ], "rhat_max": max(x["rhat"] for x in summ)}
    # cost of a full-batch delayed-acceptance step (4096 chains)
    th_full = np.exp(mu[None, :] + np.random.default_rng(5).standard_normal((C_full, 4)) @ Lc.T)
    c = rd.rd_chains_create(p, th_full, 777, step, capacity=4)
    rd.rd_chains_set_proposal(c, prop)
    rd.rd_chains_set_surrogate(c, sur)
    rd.rd_chains_run(c, 1)
    rd.rd_sync(p)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rd.rd_chains_run(c, 3)
    e1.record(stream)
    e1.synchronize()
    da_step_s = e0.elapsed_time(e1) / 1e3 / 3
    rd.rd_chains_destroy(c)
    rd.rd_surrogate_destroy(sur)
    plain_ess_s = res["plain"]["ess_per_chain_step"] * C_full / plain_step_s
    da_ess_s = res["da"]["ess_per_chain_step"] * C_full / da_step_s
    # amortised over a 5000-step run of C_full chains
    run_steps = 5000
    da_total = t_gen + t_train + run_steps * da_step_s
    out.update({
        "plain": res["plain"], "da": res["da"],
        "plain_step_s_at_full_batch": plain_step_s, "da_step_s_at_full_batch": da_step_s,
        "ess_per_s_plain": plain_ess_s, "ess_per_s_da": da_ess_s,
        "ess_per_s_da_amortised_5000_steps": res["da"]["ess_per_chain_step"] * C_full * run_steps / da_total,
        "da_vs_plain": da_ess_s / plain_ess_s,
        "method": "ESS = min over (a,b,d,gamma) of the multi-chain ESS of 152 chains x "
                  f"{steps} steps started from a pilot with an adapted proposal covariance "
                  f"(Haario et al. 2001); cost per step from {C_full}-chain steps",
        "t_wall_s": time.perf_counter() - t_total0,
    })
    return out


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
    ds = np.load(os.path.join(ROOT, "data", f"{DATASET}.npz"))
    n, C = spec["n"], args.chains
    solver = {"simt": rd.RD_SOLVER_DCT_SIMT, "tc": rd.RD_SOLVER_DCT_TC,
              "auto": rd.RD_SOLVER_AUTO}[args.solver]
    desc = rd.make_desc(2, [n], spec["tau"], spec["n_steps"], [0, 1, 2, 3],
                        [0.1, 0.9, 10.0, 200.0, 0.0], [rd.RD_PRIOR_LOGNORMAL] * 4, TRUE4,
                        [0.5] * 4, [rd.RD_STEP_LOG] * 4, solver=solver)
    stream = torch.cuda.current_stream(dev)
    p = rd.rd_problem_create(desc, stream)
    if args.kernel != "default":
        rd.rd_set_size_kernel(p, 0, KERNELS[args.kernel])
    rd.rd_set_initial_state(p, 0, ds["u0"].astype(np.float64), ds["v0"].astype(np.float64))
    rd.rd_set_observations(p, 0, ds["obs_steps"], spec["field_mask"],
                           ds["y"].astype(np.float64), spec["sigma"])
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
    times = []
    barrier()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rd.rd_chains_run(chains, 1)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    barrier()
    ck = clocks.stop()
    t_rank = float(np.sum(times))
    samples, counters = rd.rd_chains_read_samples(chains, cap, 4, C)
    solves_rank = float(counters[3]) * args.steps / (args.warmup + args.steps)
    # roofline of the solve kernel: same launch configuration, timed alone
    th = torch.tensor(samples[-1].T.copy(), dtype=torch.float64, device=dev)
    phi_d = torch.zeros(C, dtype=torch.float64, device=dev)
    st_d = torch.zeros(C, dtype=torch.int32, device=dev)
    kt = []
    for _ in range(max(1, args.kernel_reps)):
        flush.fill_(2.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rd.rd_evaluate_batch(p, th, phi_d, st_d)
        e1.record(stream)
        e1.synchronize()
        kt.append(e0.elapsed_time(e1) / 1e3)
    k_dur = float(np.mean(kt))
    # end to end: host theta in, host Phi/status out, through the C ABI
    th_h = samples[-1].T.copy()
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
        clk = ck.get("sm_mhz") or 1900.0
        kind = rd.rd_get_size_kernel(p, 0)
        if kind == rd.RD_KERNEL_SIMT:
            achieved = flop_per_solve * C / k_dur / 1e12
            fp32_peak = 152 * 128 * 2 * (ck.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp32_peak, "traffic": None,
                    "kernel": "k_solve2d_simt<128,1>", "kernel_ms": 1e3 * k_dur,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
        else:
            achieved = flop_per_solve * C / k_dur / 1e12
            tpk = _find(pk, "bf16_tflops") or FALLBACK_PEAKS["bf16_tflops"]
            kname = ("k_solve2d_tc128<2>" if kind == rd.RD_KERNEL_TC_RESIDENT
                     else "k_solve2d_tc<128>")
            roof = {"bound": "tensor", "achieved": achieved, "peak": tpk, "unit": "TFLOP/s",
                    "frac": achieved / tpk, "traffic": traffic_of(kname), "kernel": kname,
                    "kernel_ms": 1e3 * k_dur, "peak_source": f"{pk_src} bf16 burst (= fp16 rate)"}
        hbm = _find(pk, "hbm_gbs", "hbm_GBps", "copy_gbs") or FALLBACK_PEAKS["hbm_gbs"]
        roof["hbm_equiv"] = {"gbs": bytes_per_solve * C / k_dur / 1e9, "peak_gbs": hbm,
                             "frac": bytes_per_solve * C / k_dur / 1e9 / hbm,
                             "note": "16 N^2 B per proposal-step; state is resident in shared "
                                     "memory, so this is the HBM-normalised rate, not traffic"}
        line = {
            "metric": "forward solves/s (128^2, 8000 IMEX steps/solve); ESS/s in 'ess_per_s'",
            "value": value, "unit": "forward solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(C),
            "roofline": roof,
            "e2e": {"value": e2e_all, "unit": "forward solves/s",
                    "h2d_bytes_per_step": int(C * 4 * 8), "d2h_bytes_per_step": int(C * 12),
                    "call": "rd_evaluate_batch_host (host theta in, host Phi/status out)"},
            "gpu_launches": 4 * args.steps,
            "clocks": ck,
            "accept_rate": float(counters[2] / max(counters[0], 1)),
            "peaks_source": pk_src,
        }
        if not args.no_ess:
            line["ess"] = ess_comparison(rd, torch, p, stream, dev, C, t_all / args.steps)
            line["ess_per_s"] = {"plain": line["ess"]["ess_per_s_plain"],
                                 "da_surrogate": line["ess"]["ess_per_s_da"],
                                 "da_surrogate_amortised": line["ess"]["ess_per_s_da_amortised_5000_steps"]}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    rd.rd_chains_destroy(chains)
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
    ap.add_argument("--solver", default="auto", choices=["auto", "simt", "tc"])
    ap.add_argument("--kernel", default="default", choices=["default"] + sorted(KERNELS),
                    help="solve kernel of the 128^2 size (default: the library's choice)")
    ap.add_argument("--kernel-reps", type=int, default=2)
    ap.add_argument("--e2e-reps", type=int, default=1)
    ap.add_argument("--ref-sample-steps", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ess", action="store_true", help="skip the ESS/s comparison")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
