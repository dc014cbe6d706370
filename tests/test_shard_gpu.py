"""Balanced shards run one after another on one GPU (each with its own
traj_id_offset, starting on a 1024-tile chunk boundary): their chunk sums,
folded on the host in walker order, give the same bits as the unsharded
ensemble, for world sizes 2, 3 and 4."""
import numpy as np
import pytest

from paper_2608_14544_gb300 import shard
from paper_2608_14544_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch

    from paper_2608_14544_gb300 import build, qcl

    build.build()
    torch.cuda.set_device(0)
    return qcl


@pytest.mark.parametrize("cfg_id,prec", [(2, 1), (1, 0), (4, 1), (3, 1)])
def test_sharded_chunk_sums_equal_unsharded(q, cfg_id, prec):
    cfg = wl.config(cfg_id)
    steps, stride = 200, cfg["out_stride"]
    n_out = steps // stride + 1
    m = q.Model(cfg["model"])
    chunk = q.shard_chunk_walkers(m, prec)
    assert chunk == 1024 * q.shard_tile_walkers(m, prec)
    n_traj = 3 * chunk + 12_345  # four chunks, the last one ragged

    def run(first, count):
        r = q.Run(m, count, 3, prec, n_out, traj_id_offset=first)
        r.sample(cfg["init"])
        r.propagate(steps, cfg["dt"], stride)
        return r

    whole = run(0, n_traj)
    single = whole.sums()
    cs = whole.chunk_sums()
    assert cs.shape == (n_out, 4, single.shape[1])
    assert np.array_equal(shard.combine_chunks(cs), single)
    del whole
    for world in (2, 3, 4):
        parts = []
        for r in range(world):
            first, count = shard.shard_range(n_traj, world, r, chunk)
            if count:
                parts.append(run(first, count).chunk_sums())
        joined = np.concatenate(parts, axis=1)
        assert joined.shape[1] == 4
        assert np.array_equal(shard.combine_chunks(joined), single), world
