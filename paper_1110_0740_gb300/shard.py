"""Sharding of a level's patch batch over ranks, one process per GPU.

Section 4 of Mignone et al. (2012) parallelises each refinement level on its
own. It distributes the level's boxes over the processors, with the workload
of a box taken as its number of grid points (the integration costs about the
same per point). Once their ghosts are filled, the patches of one level step
are independent. So a level advance shards by patches with no exchange on the
data path. The ranks agree on the step size through one scalar reduction
(the smallest dt over the ranks; c_h follows from it), and the time of a
timed step is the slowest rank's.

The paper's balancer (CHOMBO) solves the knapsack with Kernighan-Lin.
`partition` instead deals the patches largest first to the least-loaded rank
(LPT). It then improves the split with pairwise exchanges between the most
and the least loaded rank, which is a Kernighan-Lin-style local search.
"""
from __future__ import annotations

import heapq

__all__ = ["partition", "loads", "agree_dt", "slowest"]


def partition(cells, world: int):
    """Split patches over `world` ranks by cell count.

    `cells[i]` is the workload of patch i, e.g. its interior cell count.
    Returns one sorted list of patch indices per rank. The result is
    deterministic, so every rank computes the same split, and every patch
    appears exactly once.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    cells = [int(c) for c in cells]
    if any(c < 0 for c in cells):
        raise ValueError("cell counts must be non-negative")
    order = sorted(range(len(cells)), key=lambda i: (-cells[i], i))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + cells[i], r))
    _refine(parts, cells)
    return [sorted(p) for p in parts]


def _refine(parts, cells, max_rounds: int = 64):
    """Pairwise exchanges between the most and the least loaded rank.

    Each exchange swaps one patch of the most loaded rank with one patch (or
    nothing) of the least loaded rank, picking the swap that lowers the
    larger of the two loads the most. The loop stops when no swap helps.
    """
    for _ in range(max_rounds):
        ld = [sum(cells[i] for i in p) for p in parts]
        hi = max(range(len(parts)), key=lambda r: (ld[r], -r))
        lo = min(range(len(parts)), key=lambda r: (ld[r], r))
        gap = ld[hi] - ld[lo]
        if gap <= 0:
            return
        best = None  # (new max of the pair, i, j or None)
        for i in parts[hi]:
            for j in list(parts[lo]) + [None]:
                d = cells[i] - (cells[j] if j is not None else 0)
                if 0 < d < gap:
                    m = max(ld[hi] - d, ld[lo] + d)
                    if best is None or m < best[0]:
                        best = (m, i, j)
        if best is None:
            return
        _, i, j = best
        parts[hi].remove(i)
        parts[lo].append(i)
        if j is not None:
            parts[lo].remove(j)
            parts[hi].append(j)


def loads(parts, cells):
    """Workload of each rank under a partition."""
    return [sum(int(cells[i]) for i in p) for p in parts]


def agree_dt(dt_ch, cfl: float, hmin: float, group=None):
    """Return the level step every rank takes: the smallest dt over the ranks.

    `dt_ch` is this rank's (dt, c_h) from ctu_dt on its own patches. The
    result is (dt, c_h) with c_h = C_a min dx / dt (Eq. Ca). With no process
    group, or a single rank, the local values are returned unchanged.
    """
    dt = float(dt_ch[0])
    import torch.distributed as dist
    if group is not None or (dist.is_available() and dist.is_initialized()):
        if dist.get_world_size(group) > 1:
            import torch
            t = torch.tensor([dt], dtype=torch.float64,
                             device=_reduce_device(group))
            dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
            dt = float(t.item())
    return dt, cfl * hmin / dt


def slowest(ms: float, group=None) -> float:
    """Largest per-rank step time, which is the time of the whole job."""
    import torch.distributed as dist
    if group is not None or (dist.is_available() and dist.is_initialized()):
        if dist.get_world_size(group) > 1:
            import torch
            t = torch.tensor([float(ms)], dtype=torch.float64,
                             device=_reduce_device(group))
            dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
            return float(t.item())
    return float(ms)


def _reduce_device(group):
    import torch
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")
