"""Sharding an ensemble over ranks (one GPU each): contiguous walker ranges of
2^k reduction tiles, gathered output sums combined in the library's binary
tree, which reproduces the bits of one unsharded run."""
from __future__ import annotations

import numpy as np


def shard_range(n_traj: int, world: int, rank: int, tile_walkers: int):
    """(first walker, walker count) of `rank`: every rank but the last holds the
    same power-of-two number of tiles; ranks past the end hold none."""
    n_tiles = -(-n_traj // tile_walkers)
    per = 1
    while per * world < n_tiles:
        per *= 2
    first = min(rank * per * tile_walkers, n_traj)
    last = min((rank + 1) * per * tile_walkers, n_traj)
    return first, last - first


def gather_sums(local_sums: np.ndarray, group=None) -> np.ndarray | None:
    """All ranks' output sums stacked in rank order on rank 0 (None elsewhere),
    through torch.distributed (gloo on CPU, NCCL on GPUs)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    t = torch.as_tensor(np.ascontiguousarray(local_sums, dtype=np.float64))
    backend = dist.get_backend(group)
    if backend == "nccl":
        t = t.cuda()
    out = [torch.empty_like(t) for _ in range(world)] if dist.get_rank(group) == 0 else None
    dist.gather(t, out, dst=0, group=group)
    if out is None:
        return None
    return np.stack([o.cpu().numpy() for o in out])
