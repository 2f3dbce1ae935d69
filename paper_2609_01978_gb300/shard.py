"""Sharding one aperture across processes (one GPU each).

The focal-plane field is a sum over aperture rows (Sec. 2.6: rows are
transformed in independent batches; Sec. 7.2 proposes splitting the aperture
across machines), so a rank propagates a contiguous row range and the ranks
sum their partial fields once.  The partial field is produced by a callable
(normally ``Plan.propagate_roi`` on the rank's GPU); the sum is one
``all_reduce`` of the M x M complex field over the process group (NCCL on
GPUs, gloo on CPUs).
"""
from __future__ import annotations

import math
from typing import Callable, Optional, Sequence


def chord_weights(N: int, c: int, s_R: int) -> list:
    """Samples of each row inside the aperture disc: 2 floor(sqrt(s_R - dj^2)) + 1."""
    w = []
    for j in range(N):
        dj2 = (j - c) ** 2
        w.append(0 if dj2 > s_R else 2 * math.isqrt(s_R - dj2) + 1)
    return w


def row_ranges(N: int, world: int, weights: Optional[Sequence[float]] = None) -> list:
    """Split rows [0, N) into `world` contiguous ranges of about equal total
    weight (uniform when weights is None).  Returns [(j0, j1), ...]."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if weights is None:
        return [(N * r // world, N * (r + 1) // world) for r in range(world)]
    total = float(sum(weights))
    out, j, acc = [], 0, 0.0
    for r in range(world):
        target = total * (r + 1) / world
        j0 = j
        while j < N and (acc + weights[j] <= target or r == world - 1):
            acc += weights[j]
            j += 1
        out.append((j0, j))
    out[-1] = (out[-1][0], N)
    return out


def propagate_sharded(partial: Callable[[int, int], "object"], N: int, group=None, weights=None):
    """This rank's partial field over its row range, summed over all ranks of
    `group` (torch.distributed).  Returns the full field (a torch tensor)."""
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    j0, j1 = row_ranges(N, world, weights)[rank]
    field = partial(j0, j1)
    if world > 1:
        dist.all_reduce(field, op=dist.ReduceOp.SUM, group=group)
    return field
