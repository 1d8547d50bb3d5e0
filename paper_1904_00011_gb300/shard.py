"""Parameter sets of one batch split across ranks, one process per GPU.

The live points of the nested sampler (Section 2.5) are independent problems: every set's
images, Hess diagram and likelihood depend on its own parameters and set id only (the Philox
counters carry the set id and the global pixel index), so a rank that evaluates sets
[begin, end) with ids first_set_id + begin .. gives exactly the values a single process gives
for those sets.  The only exchange is the gather of one FP64 likelihood per set at the end;
there is no collective on the data path.

Ranges are contiguous (one library call per rank, consecutive set ids) and balanced by a cost
estimate per set (pixels x draw entries).
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np


def plan(costs: Sequence[float], world: int) -> List[Tuple[int, int]]:
    """Contiguous ranges [begin, end) per rank: set k goes to the rank whose share of the total
    cost holds the midpoint of k's cost interval, so no rank exceeds total/world by more than
    one set's cost.  Empty ranges are allowed (more ranks than sets)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    c = np.asarray(costs, np.float64)
    if c.ndim != 1 or np.any(~np.isfinite(c)) or np.any(c < 0):
        raise ValueError("costs must be a 1-D array of finite non-negative numbers")
    n = c.size
    total = float(c.sum())
    if n == 0:
        return [(0, 0)] * world
    if total <= 0.0:
        c = np.ones(n)
        total = float(n)
    mid = np.cumsum(c) - 0.5 * c
    owner = np.minimum((mid / total * world).astype(np.int64), world - 1)   # non-decreasing
    return [(int(np.searchsorted(owner, r, "left")), int(np.searchsorted(owner, r, "right")))
            for r in range(world)]


def set_costs(n_ims: Sequence[int], entries: Optional[Sequence[float]] = None) -> np.ndarray:
    """Cost estimate of each set: pixels, times the set's draw entries per pixel when known."""
    px = np.asarray(n_ims, np.float64) ** 2
    if entries is None:
        return px
    return px * np.maximum(np.asarray(entries, np.float64), 1.0)


def evaluate_sharded(evaluate: Callable[[Sequence, Sequence[int], int], np.ndarray],
                     params: Sequence, n_ims: Sequence[int], first_set_id: int = 0,
                     costs: Optional[Sequence[float]] = None, group=None) -> np.ndarray:
    """Evaluate this rank's range of sets with `evaluate(params, n_ims, first_set_id)` (for a
    Simulator: a closure over Simulator.evaluate with the mock bound), then gather every set's
    likelihood on every rank.  Without an initialised process group this is one rank."""
    import torch
    import torch.distributed as dist

    distributed = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if distributed else 1
    rank = dist.get_rank(group) if distributed else 0
    n = len(params)
    if len(n_ims) != n:
        raise ValueError("params and n_ims differ in length")
    ranges = plan(set_costs(n_ims) if costs is None else costs, world)
    b, e = ranges[rank]
    mine = np.asarray(evaluate(list(params[b:e]), list(n_ims[b:e]), first_set_id + b), np.float64) \
        if e > b else np.zeros(0)
    if mine.shape != (e - b,):
        raise RuntimeError("evaluate returned %s values for %d sets" % (mine.shape, e - b))
    if world == 1:
        return mine
    # one padded FP64 row per rank; NCCL gathers device tensors, gloo host tensors
    width = max(1, max(r[1] - r[0] for r in ranges))
    dev = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")
    row = torch.full((width,), float("nan"), dtype=torch.float64, device=dev)
    row[: e - b] = torch.from_numpy(mine).to(dev)
    rows = [torch.empty_like(row) for _ in range(world)]
    dist.all_gather(rows, row, group=group)
    out = np.empty(n, np.float64)
    for r, (rb, re_) in enumerate(ranges):
        out[rb:re_] = rows[r][: re_ - rb].cpu().numpy()
    return out
