"""Sharding an ensemble over ranks (one GPU each) with the bits of one
unsharded run.

The reduction tree sums 256-walker tiles (64 or 128 for split many-mode and
N-state kernels) by a zero-padded binary tree in walker order, computed in
blocks of 1024 tiles.  A chunk of 1024 tiles is therefore an aligned subtree:
a rank whose walkers start at a chunk boundary computes each of its chunks'
sums exactly as the unsharded run does (qcl_read_chunk_sums), and the binary
tree over all chunks in walker order (qcl_combine_shards) gives the unsharded
rows.  Ranks take contiguous runs of floor(C / world) or ceil(C / world) of
the C chunks, so their walker counts differ by at most one chunk.
"""
from __future__ import annotations

import numpy as np


def chunk_bounds(n_chunks: int, world: int, rank: int):
    """[first chunk, end chunk) of `rank` (balanced contiguous runs)."""
    return rank * n_chunks // world, (rank + 1) * n_chunks // world


def shard_range(n_traj: int, world: int, rank: int, chunk_walkers: int):
    """(first walker, walker count) of `rank` for chunks of chunk_walkers
    walkers (qcl_shard_chunk_walkers)."""
    n_chunks = -(-n_traj // chunk_walkers)
    c0, c1 = chunk_bounds(n_chunks, world, rank)
    first = min(c0 * chunk_walkers, n_traj)
    last = min(c1 * chunk_walkers, n_traj)
    return first, last - first


def gather_chunk_sums(local: np.ndarray, n_traj: int, chunk_walkers: int,
                      group=None) -> np.ndarray | None:
    """All ranks' chunk sums ([rows, local chunks, q]) joined in walker order on
    rank 0 as [rows, chunks, q] (None elsewhere), through torch.distributed
    (gloo on CPU, NCCL on GPUs).  Ranks send equal-sized, zero-padded blocks."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n_chunks = -(-n_traj // chunk_walkers)
    cmax = -(-n_chunks // world)
    rows, own, q = local.shape
    pad = np.zeros((rows, cmax, q))
    pad[:, :own] = local
    t = torch.as_tensor(pad)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.empty_like(t) for _ in range(world)] if dist.get_rank(group) == 0 else None
    dist.gather(t, out, dst=0, group=group)
    if out is None:
        return None
    parts = []
    for r in range(world):
        c0, c1 = chunk_bounds(n_chunks, world, r)
        parts.append(out[r].cpu().numpy()[:, :c1 - c0])
    return np.concatenate(parts, axis=1)


def combine_chunks(chunk_sums: np.ndarray) -> np.ndarray:
    """Rows [rows, q] from the chunk sums of every shard ([rows, chunks, q],
    chunks in walker order): the library's zero-padded binary tree over the
    chunks, which reproduces the unsharded fold."""
    from . import qcl

    rows, n_chunks, q = chunk_sums.shape
    by_chunk = np.ascontiguousarray(np.moveaxis(chunk_sums, 1, 0).reshape(n_chunks, rows * q))
    return qcl.combine_shards(by_chunk).reshape(rows, q)
