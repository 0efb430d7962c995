"""Independent graph pairs spread over several GPUs, one process per GPU.

Pairs of a batch are independent problems, so they shard with no exchange
on the data path: every rank solves its own share with
``Solver.match_batched`` and the permutations and statistics are gathered
once at the end.  A single pair does not shard (every P1/P2 round of Eq. P1
needs the global column sums of Y), so one pair runs on one GPU.

The share of each rank is a longest-processing-time partition of the pairs'
estimated costs: per outer iteration the gradient A X A' costs
2 N m (N + m) flops (Section 4.1) and the projection runs up to I_1 rounds
over the N x N slacked matrix (Section 4.3).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Sequence

import numpy as np


def pair_cost(n_a: int, n_b: int, max_inner: int = 1000, flops_per_entry_round: float = 400.0) -> float:
    """Relative cost of one outer iteration of a pair with n_a and n_b nodes:
    the gradient's flops plus the projection's entry-rounds weighted as
    ``flops_per_entry_round`` flops each (a round is latency- and
    bandwidth-bound, not flop-bound)."""
    N, m = max(n_a, n_b), min(n_a, n_b)
    return 2.0 * N * m * (N + m) + flops_per_entry_round * max_inner * N * N


def partition(costs: Sequence[float], world: int) -> list[list[int]]:
    """Longest-processing-time assignment of items to `world` ranks: items in
    decreasing cost (ties by index) go to the least-loaded rank (ties by rank
    index).  Deterministic, so every rank computes the same partition without
    communicating.  Each rank's list is in increasing item order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    shares: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i)):
        r = min(range(world), key=lambda r: (load[r], r))
        shares[r].append(i)
        load[r] += float(costs[i])
    return [sorted(s) for s in shares]


@dataclass
class ShardResult:
    index: int          # position of the pair in the global list
    rank: int           # rank that solved it
    perm: np.ndarray    # int32, n_a entries (caller orientation), -1 = unmatched
    stats: dict


def solve_sharded(solve: Callable[[list], list], pairs: Sequence, shapes: Sequence[tuple[int, int]],
                  rank: int, world: int, gather: Callable[[object], list] | None = None,
                  max_inner: int = 1000) -> list[ShardResult]:
    """Solves this rank's share of `pairs` with `solve` (for example
    ``lambda ps: solver.match_batched(ps, params)``) and returns every
    pair's result, in the global order, on every rank.

    shapes[i] = (n_a, n_b) of pair i.  `gather(obj)` returns the list of all
    ranks' objects (``torch.distributed.all_gather_object``); it is the only
    collective and runs once, after the solves."""
    shares = partition([pair_cost(a, b, max_inner) for a, b in shapes], world)
    mine = shares[rank]
    local = []
    if mine:
        outs = solve([pairs[i] for i in mine])
        for i, o in zip(mine, outs):
            st = o.stats
            stats = {k: getattr(st, k) for k, _ in getattr(st, "_fields_", [])} if hasattr(st, "_fields_") \
                else dict(st)
            perm = o.perm.cpu().numpy() if hasattr(o.perm, "cpu") else np.asarray(o.perm)
            local.append(ShardResult(i, rank, perm.astype(np.int32), stats))
    parts = gather(local) if gather is not None else [local]
    out: list[ShardResult | None] = [None] * len(pairs)
    for part in parts:
        for r in part:
            if out[r.index] is not None:
                raise RuntimeError(f"pair {r.index} solved twice")
            out[r.index] = r
    missing = [i for i, r in enumerate(out) if r is None]
    if missing:
        raise RuntimeError(f"pairs {missing} were not solved by any rank")
    return out  # type: ignore[return-value]


def torch_gather(obj):
    """all_gather_object over the default process group."""
    import torch.distributed as dist
    res = [None] * dist.get_world_size()
    dist.all_gather_object(res, obj)
    return res
