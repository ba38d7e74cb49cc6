"""Multi-GPU host logic: one process per GPU, pairs sharded across ranks.

Pair tests are independent (the method has no exchange step), so several
GPUs split a batch by pairs with no collective on the data path: every rank
computes the same deterministic assignment, packs and tests its own pairs on
its own GPU, and the per-pair results are gathered once at the end.  The only
collectives are the result gather and the max-over-ranks timing.
"""
from __future__ import annotations

import numpy as np


def shard(n, m, world: int):
    """Longest-first greedy assignment of pairs to `world` ranks by their
    size N = n + m (the work of a pair grows with N): every rank gets the
    same answer.  Returns one sorted index array per rank."""
    n = np.asarray(n, dtype=np.int64)
    m = np.asarray(m, dtype=np.int64)
    cost = n + m
    order = np.argsort(-cost, kind="stable")
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(len(cost), dtype=np.int64)
    for p in order:
        r = int(np.argmin(load))  # lowest load, lowest rank on ties
        owner[p] = r
        load[r] += cost[p]
    return [np.nonzero(owner == r)[0] for r in range(world)]


def offsets(n, m):
    n = np.asarray(n, dtype=np.int64)
    m = np.asarray(m, dtype=np.int64)
    off = np.zeros(len(n) + 1, dtype=np.int64)
    np.cumsum(n + m, out=off[1:])
    return off


def pack(XY, n, m, idx):
    """Rows of the pairs `idx` of a packed batch (X rows then Y rows per pair),
    as a new packed batch.  XY is a numpy array or a torch tensor."""
    off = offsets(n, m)
    rows = np.concatenate([np.arange(off[p], off[p + 1]) for p in idx]) if len(idx) else np.zeros(0, np.int64)
    if hasattr(XY, "index_select"):
        import torch

        sub = XY.index_select(0, torch.from_numpy(rows).to(XY.device))
    else:
        sub = XY[rows]
    return sub, np.asarray(n)[idx], np.asarray(m)[idx]


def gather(idx, results, P: int, group=None):
    """All ranks' per-pair results, in pair order, on every rank."""
    import torch.distributed as dist

    mine = list(zip([int(i) for i in idx], results))
    everyone = [None] * dist.get_world_size(group)
    dist.all_gather_object(everyone, mine, group=group)
    out = [None] * P
    for part in everyone:
        for i, r in part:
            out[i] = r
    if any(r is None for r in out):
        raise RuntimeError("a pair has no result after the gather")
    return out


def max_over_ranks(seconds: float, device=None, group=None) -> float:
    """The slowest rank's time (the job's time)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def run_sharded(runner, XY, n, m, rank: int, world: int, group=None):
    """Tests this rank's share of the batch with `runner(XY_sub, n_sub, m_sub)`
    (a list of per-pair results) and returns every pair's result."""
    idx = shard(n, m, world)[rank]
    sub, ns, ms = pack(XY, n, m, idx)
    res = runner(sub, ns, ms) if len(idx) else []
    return gather(idx, res, len(n), group=group)
