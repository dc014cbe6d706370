"""Sharding over ranks on CPU (gloo, world sizes 2, 3, 4 and 8): the partition
gives each rank a contiguous run of 1024-tile chunks, within one chunk of the
others, and gathering the ranks' chunk sums and folding them in walker order
reproduces, bit for bit, the binary reduction tree over all tiles of one
unsharded ensemble."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2608_14544_gb300 import shard

CHUNK_TILES = 1024


def tree_over_tiles(parts):
    """Zero-padded binary tree over the first axis (the unsharded fold)."""
    n = parts.shape[0]
    p2 = 1
    while p2 < n:
        p2 *= 2
    lev = np.zeros((p2,) + parts.shape[1:])
    lev[:n] = parts
    while lev.shape[0] > 1:
        lev = lev[0::2] + lev[1::2]
    return lev[0]


def chunk_sums(parts):
    """The fold's first level: a binary tree over each 1024-tile block."""
    n = parts.shape[0]
    return np.stack([tree_over_tiles(np.concatenate(
        [parts[c:c + CHUNK_TILES], np.zeros((max(0, c + CHUNK_TILES - n),) + parts.shape[1:])]))
        for c in range(0, n, CHUNK_TILES)])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_traj, tile, q, rows, out_dir):
    import torch.distributed as dist

    from paper_2608_14544_gb300 import qcl

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    rng = np.random.default_rng(123)
    n_tiles = -(-n_traj // tile)
    # per-tile partials of `rows` output times, over many orders of magnitude
    parts = rng.normal(size=(n_tiles, rows, q)) * np.exp(rng.normal(size=(n_tiles, 1, 1)) * 4)
    chunk_walkers = CHUNK_TILES * tile
    first, count = shard.shard_range(n_traj, world, rank, chunk_walkers)
    t0, t1 = first // tile, -(-(first + count) // tile)
    local = (np.moveaxis(chunk_sums(parts[t0:t1]), 0, 1) if count > 0
             else np.zeros((rows, 0, q)))
    gathered = shard.gather_chunk_sums(local, n_traj, chunk_walkers)
    if rank == 0:
        qcl.load()
        np.save(os.path.join(out_dir, "combined.npy"), shard.combine_chunks(gathered))
        np.save(os.path.join(out_dir, "single.npy"), tree_over_tiles(parts))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_traj", [(2, 256 * 1024 * 5 + 77), (3, 256 * 1024 * 7 + 1),
                                          (4, 256 * 1024 * 4), (8, 256 * 1024 * 13 + 300),
                                          (4, 300)])
def test_gloo_shards_combine_bitwise(tmp_path, world, n_traj):
    from paper_2608_14544_gb300 import build

    build.build()
    mp.spawn(_worker, args=(world, _free_port(), n_traj, 256, 32, 3, str(tmp_path)),
             nprocs=world, join=True)
    c = np.load(tmp_path / "combined.npy")
    s = np.load(tmp_path / "single.npy")
    assert np.array_equal(c, s)


def test_partition_is_balanced_aligned_and_complete():
    for chunk in (1024 * 256, 1024 * 64):
        for n_traj in (1, 255, chunk - 1, chunk, chunk + 1, 10_000_000, 100_000_000):
            n_chunks = -(-n_traj // chunk)
            for world in (1, 2, 3, 4, 8):
                got = [shard.shard_range(n_traj, world, r, chunk) for r in range(world)]
                assert sum(c for _, c in got) == n_traj
                end = 0
                for f, c in got:  # contiguous, in rank order, starting on chunk boundaries
                    assert f == end and (c == 0 or f % chunk == 0)
                    end = f + c
                per = [-(-c // chunk) for _, c in got]
                assert max(per) - min(per) <= 1
                assert sum(per) == n_chunks
    # the benchmark's size over 8 ranks: within one chunk (2.6 %) of balance
    counts = [shard.shard_range(10_000_000, 8, r, 1024 * 256)[1] for r in range(8)]
    assert max(counts) <= 1.06 * 10_000_000 / 8 and min(counts) > 0
