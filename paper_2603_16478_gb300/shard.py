"""Independent scenes of a batch shared out across ranks, one process per GPU.

The one-step adjoint of a scene is self-contained, so a batch of scenes splits across GPUs with no
exchange during the solve (the paper runs on one GPU; a single scene's triangular solves and
Krylov dot products are global and are not split).  Each rank solves its shard of scenes as one
batched call; afterwards the per-scene results are gathered on every rank, and parameter
gradients shared by all scenes are summed with one all-reduce.

Shards are planned by LPT (longest processing time first): scenes sorted by estimated cost,
each given to the least loaded rank.  A rank whose own work fails reports the scenes it lost
instead of results, so the others learn which scenes are missing at the gather; a rank that
disappears makes the others' next collective fail with an error (the process group's timeout).
Only host-side plumbing lives here: every numeric step runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import torch
import torch.distributed as dist


def scene_cost(n_verts: int, nnz_L: int, n_contacts: int, iterations: float = 50.0) -> float:
    """Relative cost of one scene's adjoint: Krylov iterations x (factor + vector traffic) plus
    the dense capacitance inverse, (3 n_c)^3."""
    return iterations * (12.0 * nnz_L + 24.0 * 3 * n_verts) + (3.0 * n_contacts) ** 3 / 64.0


def plan_shards(costs: Sequence[float], world_size: int) -> List[List[int]]:
    """LPT assignment of items to ranks: items by decreasing cost (ties: lower index first), each
    to the rank with the smallest load so far (ties: lower rank).  Every item appears once; each
    rank's list is in increasing item order."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world_size
    shards: List[List[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += float(costs[i])
    return [sorted(s) for s in shards]


class ShardLost(RuntimeError):
    """Some scenes have no result: their rank failed, or a rank left the group."""

    def __init__(self, message: str, missing: Sequence[int] = ()):
        super().__init__(message)
        self.missing = list(missing)


@dataclass
class ShardResult:
    """What one rank contributes at the gather."""
    rank: int
    items: List[int]
    results: Dict[int, object] = field(default_factory=dict)
    error: Optional[str] = None


def run_sharded(costs: Sequence[float], run_shard: Callable[[List[int]], Dict[int, object]],
                group=None, raise_on_loss: bool = True):
    """Run ``run_shard`` on this rank's shard and gather every rank's results.

    ``run_shard(items) -> {item: result}`` solves the given scenes (one batched call).  Returns
    (results for all items, shards).  If a rank's ``run_shard`` raised, its items are missing:
    with ``raise_on_loss`` every rank raises ShardLost naming them, otherwise the partial results
    are returned.  A rank that left the group makes the gather raise on the others."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    shards = plan_shards(costs, world)
    mine = shards[rank]
    out = ShardResult(rank, mine)
    try:
        out.results = dict(run_shard(mine)) if mine else {}
    except Exception as e:  # noqa: BLE001 -- reported to every rank at the gather
        out.error = f"{type(e).__name__}: {e}"
    if world > 1:
        gathered: List[Optional[ShardResult]] = [None] * world
        dist.all_gather_object(gathered, out, group=group)
    else:
        gathered = [out]
    results: Dict[int, object] = {}
    missing: List[int] = []
    errors = []
    for g in gathered:
        if g.error is not None:
            missing += g.items
            errors.append(f"rank {g.rank}: {g.error}")
        else:
            results.update(g.results)
    missing = sorted(set(missing) | (set(range(len(costs))) - set(results)))
    if missing and raise_on_loss:
        raise ShardLost("; ".join(errors) or "results missing", missing)
    return results, shards


def allreduce_shared(grad: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of a parameter gradient shared by all scenes (one all-reduce, in place)."""
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad
