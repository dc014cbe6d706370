"""Sharding over ranks on CPU (gloo, world sizes 2 and 4): the partition is a
set of aligned power-of-two tile ranges, and gathering the shards' sums and
combining them reproduces, bit for bit, the binary reduction tree over all
tiles of one unsharded ensemble."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2608_14544_gb300 import shard


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


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_traj, tile, q, out_dir):
    import torch.distributed as dist

    from paper_2608_14544_gb300 import qcl

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    rng = np.random.default_rng(123)
    n_tiles = -(-n_traj // tile)
    parts = rng.normal(size=(n_tiles, q)) * np.exp(rng.normal(size=(n_tiles, 1)) * 4)
    first, count = shard.shard_range(n_traj, world, rank, tile)
    t0, t1 = first // tile, -(-(first + count) // tile)
    local = tree_over_tiles(parts[t0:t1]) if count > 0 else np.zeros(q)
    gathered = shard.gather_sums(local)
    if rank == 0:
        qcl.load()
        combined = qcl.combine_shards(gathered)
        np.save(os.path.join(out_dir, "combined.npy"), combined)
        np.save(os.path.join(out_dir, "single.npy"), tree_over_tiles(parts))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_traj", [(2, 256 * 37 + 5), (4, 256 * 1000 + 1), (4, 300)])
def test_gloo_shards_combine_bitwise(tmp_path, world, n_traj):
    from paper_2608_14544_gb300 import build

    build.build()
    mp.spawn(_worker, args=(world, _free_port(), n_traj, 256, 32, str(tmp_path)), nprocs=world,
             join=True)
    c = np.load(tmp_path / "combined.npy")
    s = np.load(tmp_path / "single.npy")
    assert np.array_equal(c, s)


def test_partition_is_aligned_and_complete():
    for n_traj in (1, 255, 256, 257, 10_000, 1_000_000):
        for world in (1, 2, 3, 4, 8):
            got = [shard.shard_range(n_traj, world, r, 256) for r in range(world)]
            assert sum(c for _, c in got) == n_traj
            per = None
            for r, (f, c) in enumerate(got):
                if c == 0:
                    continue
                assert f % 256 == 0
                tiles = -(-c // 256)
                if f + c < n_traj:  # all but the last holder: the same power of two
                    assert tiles & (tiles - 1) == 0
                    per = per or tiles
                    assert tiles == per and (f // 256) % tiles == 0
