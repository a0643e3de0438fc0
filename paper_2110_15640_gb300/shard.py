"""Splitting the photon-transport work over several GPUs (one process per GPU).

Jobs (wavelength, g-ordinate, phase) and packet ranges are independent: every packet draws its
random numbers from Philox keyed by (seed; packet, event, job key), so a packet gives the same
contribution on any rank.  The only exchange a sharded run needs is a sum of per-job tallies, done
on 64-bit fixed-point integers (2^-32 resolution, the same representation the kernels accumulate
in), so the reduced result is exact and independent of the rank order.  The benchmark's weak-scaling
runs use no collective in the data path at all: each rank processes its own copy of the workload.
"""
from __future__ import annotations

FIX_SCALE = 4294967296.0   # 2^32


def rank_seed(seed: int, rank: int) -> int:
    """Distinct packet streams per rank for weak scaling (a large odd stride keeps seeds apart)."""
    return int(seed) + 7919 * int(rank)


def split_jobs(n_jobs: int, rank: int, world: int):
    """Round-robin job indices of `rank` (spreads heavy and light jobs alike)."""
    return list(range(rank, n_jobs, world))


def split_packets(n_packets: int, rank: int, world: int):
    """Contiguous packet block (packet0, n_run) of `rank`; blocks cover 0..n_packets-1 exactly once."""
    base, extra = divmod(int(n_packets), int(world))
    packet0 = rank * base + min(rank, extra)
    return packet0, base + (1 if rank < extra else 0)


def to_fixed(values):
    """Per-packet contributions to 64-bit fixed point (round to nearest), as the kernels do."""
    import numpy as np
    return np.rint(np.asarray(values, dtype=np.float64) * FIX_SCALE).astype(np.int64)


def reduce_fixed(local_sum, group=None):
    """Exact cross-rank sum of int64 fixed-point tallies (torch.distributed all_reduce)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(local_sum, dtype=torch.int64).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def max_over_ranks(seconds: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
