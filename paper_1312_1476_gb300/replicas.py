"""Host-side logic for running the sampler as independent replicas, one per
GPU and process (torch.distributed ranks).

Samples, Hutchinson probes and requests are independent Lanczos runs
(Section 6: each probe term is computed on its own), so N GPUs work on disjoint
shares with no device-side exchange.  The only cross-rank steps are host-side:
the maximum of the ranks' timings, and combining the per-probe log-det terms
of all replicas into one estimate and standard error.
"""
from __future__ import annotations

import numpy as np


def shard(count: int, rank: int, world: int):
    """[start, stop) of `count` units owned by `rank` (contiguous, balanced)."""
    base, extra = divmod(int(count), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def replica_seed(seed: int, rank: int) -> int:
    """Distinct Philox keys per replica (the library's counters already index
    vectors inside one call)."""
    return (int(seed) + 0x9E3779B97F4A7C15 * int(rank)) & 0xFFFFFFFFFFFFFFFF


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar (the timed region's device time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine_logdet(q_local, shift: float, dist=None):
    """Hutchinson estimate from the per-probe terms of all replicas:
    (mean_i q_i + shift, sd(q_i) / sqrt(N)) over the N probes of all ranks."""
    q = np.asarray(q_local, dtype=np.float64).reshape(-1)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, q.tolist())
        q = np.concatenate([np.asarray(p, dtype=np.float64) for p in parts])
    n = q.size
    est = float(q.mean()) + float(shift)
    se = float(q.std(ddof=1) / np.sqrt(n)) if n > 1 else float("nan")
    return est, se, n
