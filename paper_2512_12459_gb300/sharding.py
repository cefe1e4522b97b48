"""Data-parallel sharding of the training step, one GPU per rank.

The field and its index are replicated on every rank and the hit points are
split by view. The forward needs no communication. The loss is the MSE over
the visible points of all views together (Sec. 4.3: one mean over the set V
of supervised points), so a rank whose MSE gradient g_r is normalised by its
own valid count |V_r| contributes (|V_r| / |V|) g_r to the gradient of the
global loss: the per-Gaussian gradients are scaled by that weight and summed
with one all-reduce per tensor, after which every rank applies the same Adam
step to its replica. Timings are combined as the maximum over ranks.

Everything here is host-side glue around torch.distributed; the per-rank
work runs in libgpf.
"""

from __future__ import annotations

from typing import List, Optional, Sequence

import torch
import torch.distributed as dist


def shard_views(view_sizes: Sequence[int], world: int, rank: int) -> List[int]:
    """Indices of the views rank `rank` of `world` processes.

    Greedy balance by hit-point count: views in decreasing size (ties by
    index) each go to the rank with the fewest hit points so far (ties by
    rank). Deterministic, so every rank computes the same assignment without
    communication. Returned in increasing view order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of world {world}")
    load = [0] * world
    owner = [0] * len(view_sizes)
    for v in sorted(range(len(view_sizes)), key=lambda i: (-int(view_sizes[i]), i)):
        r = min(range(world), key=lambda j: (load[j], j))
        owner[v] = r
        load[r] += int(view_sizes[v])
    return [v for v in range(len(view_sizes)) if owner[v] == rank]


def global_count(n_local: int, device=None, group=None) -> int:
    """Sum over ranks of an integer (the valid hit points of every rank)."""
    if not (dist.is_available() and dist.is_initialized()):
        return int(n_local)
    t = torch.tensor([int(n_local)], dtype=torch.int64, device=device)
    dist.all_reduce(t, group=group)
    return int(t.item())


def allreduce_gradients(grads: Sequence[torch.Tensor], n_local: int, n_total: int,
                        group=None) -> None:
    """In place: grads <- sum over ranks of (n_local / n_total) * grads, the
    gradient of the MSE over all ranks' valid points when each rank's grads
    come from its own MSE normalised by n_local."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return
    w = 0.0 if n_total == 0 else float(n_local) / float(n_total)
    for t in grads:
        if w != 1.0:
            t.mul_(w)
        dist.all_reduce(t, group=group)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The maximum of a float over ranks (step times)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(value: float, device=None, group=None) -> float:
    """The sum of a float over ranks (hit points processed)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, group=group)
    return float(t.item())


def init_from_env(backend: str, device: Optional[torch.device] = None) -> None:
    """init_process_group from the torchrun environment (RANK, WORLD_SIZE,
    MASTER_ADDR, MASTER_PORT)."""
    if device is not None and backend == "nccl":
        dist.init_process_group(backend, device_id=device)
    else:
        dist.init_process_group(backend)
