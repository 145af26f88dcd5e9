"""Per-size choice of the solve kernel, measured and persisted.

Uneven batching puts proposals of several grid sizes into one evaluation; each
size runs the kernel that a timed search found fastest on this GPU for that
size (``rd_autotune`` in the C library: every applicable kernel solves the same
probe batch, CUDA-event timed, median of the trials).  The choices are kept in
a small JSON file keyed by GPU name, dimension, grid size and IMEX step count,
so later runs on the same kind of GPU reuse them without re-timing.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import (RD_KERNEL_CG, RD_KERNEL_SIMT, RD_KERNEL_TC_RESIDENT, RD_KERNEL_TC_STACKED,
               rd_autotune, rd_get_size_kernel, rd_get_size_schedule, rd_set_size_kernel,
               rd_set_size_schedule)

KERNEL_NAMES = {RD_KERNEL_SIMT: "simt", RD_KERNEL_TC_STACKED: "tc_stacked",
                RD_KERNEL_TC_RESIDENT: "tc_resident", RD_KERNEL_CG: "cg"}
_BY_NAME = {v: k for k, v in KERNEL_NAMES.items()}
_COLUMNS = (RD_KERNEL_SIMT, RD_KERNEL_TC_STACKED, RD_KERNEL_TC_RESIDENT, RD_KERNEL_CG)


def cache_key(gpu: str, dim: int, n: int, n_steps: int) -> str:
    return f"{gpu}|{dim}d|n={n}|steps={n_steps}"


def fastest(times_row) -> int:
    """Kernel with the lowest finite time in one row of rd_autotune's output."""
    best, best_t = None, math.inf
    for kind, t in zip(_COLUMNS, times_row):
        if t is not None and math.isfinite(t) and t < best_t:
            best, best_t = kind, t
    if best is None:
        raise ValueError("no kernel has a finite time")
    return best


def load_table(path: str | None) -> dict:
    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def save_table(path: str, table: dict) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(p, gpu: str, dim: int, sizes, n_steps: int, theta, cache_path: str | None = None,
         n_trials: int = 3, probe_steps: int = 200, force: bool = False) -> dict:
    """Sets the kernel and schedule (persistent CTAs per SM) of every size of
    problem ``p`` (grid sizes ``sizes``, in size-index order) from the cache
    at ``cache_path`` when it has all of them, else by ``rd_autotune`` on the
    probe batch ``theta`` (host [B][n_params]) and writes the result back.
    Returns {size_idx: entry}."""
    table = load_table(cache_path)
    keys = [cache_key(gpu, dim, n, n_steps) for n in sizes]
    if not force and all(k in table for k in keys):
        for s, k in enumerate(keys):
            rd_set_size_kernel(p, s, _BY_NAME[table[k]["kernel"]])
            rd_set_size_schedule(p, s, int(table[k].get("ctas_per_sm", 0)))
        return {s: dict(table[k], cached=True) for s, k in enumerate(keys)}
    times = rd_autotune(p, np.asarray(theta, dtype=np.float64), n_trials=n_trials,
                        probe_steps=probe_steps, n_sizes=len(sizes))
    out = {}
    for s, (n, k) in enumerate(zip(sizes, keys)):
        kind = rd_get_size_kernel(p, s)
        assert kind == fastest(times[s])
        entry = {"kernel": KERNEL_NAMES[kind], "ctas_per_sm": int(rd_get_size_schedule(p, s)),
                 "n": int(n), "probe_steps": int(probe_steps),
                 "seconds_per_proposal": {KERNEL_NAMES[c]: (None if not math.isfinite(t) else t)
                                          for c, t in zip(_COLUMNS, times[s])}}
        table[k] = entry
        out[s] = dict(entry, cached=False)
    if cache_path:
        save_table(cache_path, table)
    return out
