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


def merge_best_device(record, collides, offset: int, group=None):
    """The same merge with every step on the tensors' device and no host
    synchronisation, for use inside a stream of queued work.

    record: the rank's local best as the 36-float selection record (index,
    cost, residual, then the 33 coefficients c_x, c_y, c_psi), e.g. what
    am_get_best_async writes to device memory; collides: a one-element bool
    or float tensor (the record's trajectory collides); offset: the global
    index of the rank's first trajectory.  Every rank gathers every rank's
    key and coefficients in one all-gather and takes the lexicographically
    smallest key (collision-free first, then cost, then global index; a
    non-finite cost ranks last).  Returns the winner as a 36-float record on
    the same device, its index global."""
    world = dist.get_world_size(group)
    rec = record.reshape(36).to(torch.float64)
    col = collides.reshape(1).to(torch.float64)
    cost = rec[1:2]
    flag = torch.where(torch.isfinite(cost), col, torch.full_like(col, 2.0))
    row = torch.cat([flag, torch.nan_to_num(cost, nan=float("inf")), rec[0:1] + float(offset), rec[1:36]])
    rows = [torch.empty_like(row) for _ in range(world)]
    dist.all_gather(rows, row, group=group)
    table = torch.stack(rows)                       # [world, 38]: flag, cost, gidx, cost, residual, coeffs
    inf = torch.full_like(table[:, 0], float("inf"))
    m = table[:, 0] == table[:, 0].min()
    c = torch.where(m, table[:, 1], inf)
    m = m & (table[:, 1] == c.min())
    w = torch.argmin(torch.where(m, table[:, 2], inf))
    win = table[w]
    return torch.cat([win[2:3], win[3:5], win[5:38]]).to(record.dtype)
