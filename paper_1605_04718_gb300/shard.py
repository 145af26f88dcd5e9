"""Chains split over processes, one process per GPU.

The chains of Sec. 2.1 are independent, so a run with several GPUs gives each
process a contiguous range of them; with ``rd_chains_set_first_chain`` set to
the range's start and the same seed everywhere, every chain draws the same
random numbers it would draw in a one-process run.  Nothing is exchanged while
sampling; afterwards the samples (or any per-process result) are gathered and
pooled, and throughput is the units of all processes over the slowest one's
time.  The collectives go through ``torch.distributed`` (NCCL between GPUs,
gloo on the host).
"""
from __future__ import annotations

import numpy as np


def shard(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """(first, count) of this rank's contiguous range of n_total chains; the
    counts differ by at most one, lower ranks take the extra chains."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_total >= 0")
    base, extra = divmod(n_total, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def gather_chains(local, dist=None, group=None):
    """Samples [steps][P][C_rank] of every rank, concatenated along the chain
    axis in rank order (so in global chain order); returned on every rank.
    With ``dist`` None (one process) the input is returned."""
    local = np.asarray(local)
    if dist is None or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return local
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, local, group=group)
    return np.concatenate(parts, axis=-1)


def aggregate_rate(units_local: float, seconds_local: float, dist=None, group=None):
    """(units of all ranks, max seconds over ranks, units / seconds): the
    whole-job rate, timed by the slowest rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return units_local, seconds_local, units_local / seconds_local
    vals = [None] * dist.get_world_size(group)
    dist.all_gather_object(vals, (float(units_local), float(seconds_local)), group=group)
    units = sum(v[0] for v in vals)
    secs = max(v[1] for v in vals)
    return units, secs, units / secs
