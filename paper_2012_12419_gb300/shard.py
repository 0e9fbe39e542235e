"""Host-side sharding of a batch of independent instances across ranks.

The instances of the batched workload are independent MDPs, so a multi-GPU run splits
them across ranks with no exchange on the data path: each rank builds and solves its own
sub-batch, and only the per-instance results are gathered at the end.  The split is the
longest-processing-time-first rule (largest estimated cost to the least-loaded rank),
whose makespan is within 4/3 of the optimum.

The cost of an instance is its work to the 1e-6 residual: successor updates per sweep
(S x A x (2H + 3), the padded row bound) times the sweeps a gamma-contraction needs to
shrink the first residual to the tolerance.
"""
from __future__ import annotations

import heapq
import math


def instance_cost(p: dict, tol: float = 1e-6) -> float:
    H, C, Q, g = int(p["H"]), int(p["C"]), int(p["Q"]), float(p["gamma"])
    S = 2 * (Q + 1) * (C + 1) ** H
    per_sweep = S * (H + 1) * (2 * H + 3)
    # first residual ~ max |R| ~ C H; sweeps until gamma^k C H < tol (1 - gamma)
    sweeps = max(1.0, math.log(tol * (1.0 - g) / max(1.0, C * H)) / math.log(g))
    return per_sweep * sweeps


def lpt_shards(costs, n_ranks: int):
    """Index lists, one per rank, from the LPT rule; each list is in ascending index order."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(n_ranks)]
    shards = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in shards]


def shard_of(params_list, rank: int, world: int, tol: float = 1e-6):
    """This rank's instance indices and parameter dicts."""
    idx = lpt_shards([instance_cost(p, tol) for p in params_list], world)[rank]
    return idx, [params_list[i] for i in idx]


def gather_by_index(local: dict, n: int, group=None) -> list:
    """Collect {instance index: result} from every rank into one list of length n
    (torch.distributed object gather, after the timed work)."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    out = [None] * n
    for part in parts:
        for i, v in part.items():
            if out[i] is not None:
                raise RuntimeError(f"instance {i} solved on two ranks")
            out[i] = v
    missing = [i for i, v in enumerate(out) if v is None]
    if missing:
        raise RuntimeError(f"instances {missing[:8]} solved on no rank")
    return out
