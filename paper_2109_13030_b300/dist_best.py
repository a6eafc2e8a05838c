"""Cross-rank best-trajectory merge for a batch sharded over several GPUs.

Trajectories of one planning problem are independent (Sec. III-D runs the
same AM loop on every sample), so a batch splits into contiguous ranges, one
per rank, with no exchange during the iterations.  The one exchange is the
final selection of the best trajectory over all ranks: each rank contributes
its local best as a key (collides, cost, global index), the smallest key
wins in lexicographic order (a collision-free trajectory first, then the
lowest cost, then the lowest index), and the winner's 33 coefficients are
broadcast from the rank that owns them.

Works with any torch.distributed backend; the tensors live on `device`
(a CUDA device under NCCL, the CPU under gloo).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(B_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [first, last) range of trajectories owned by a rank."""
    lo = B_total * rank // world
    hi = B_total * (rank + 1) // world
    return lo, hi


def key_of(collides: bool, cost: float, global_index: int) -> tuple:
    return (1 if collides else 0, float(cost), int(global_index))


def merge_best(collides: bool, cost: float, global_index: int, coeffs, device, group=None) -> dict:
    """All ranks call this with their local best; all return the global best
    as dict(coeffs (3 x 11 float32 tensor), cost, index, collides, rank)."""
    world = dist.get_world_size(group)
    mine = torch.tensor([1.0 if collides else 0.0, float(cost), float(global_index)],
                        dtype=torch.float64, device=device)
    keys = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(keys, mine, group=group)
    table = [(int(k[0].item()), float(k[1].item()), int(k[2].item()), r) for r, k in enumerate(keys)]
    flag, best_cost, best_idx, owner = min(table)
    buf = torch.as_tensor(coeffs, dtype=torch.float32).reshape(33).to(device).clone()
    dist.broadcast(buf, src=dist.get_global_rank(group, owner) if group is not None else owner,
                   group=group)
    return dict(coeffs=buf.reshape(3, 11), cost=best_cost, index=best_idx, collides=bool(flag),
                rank=owner)
