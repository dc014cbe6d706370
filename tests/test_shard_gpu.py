"""Shards run one after another on one GPU (each with its own traj_id_offset)
and combined on the host give the same bits as the unsharded ensemble."""
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


@pytest.mark.parametrize("cfg_id,prec", [(2, 1), (1, 0), (4, 1)])
def test_sharded_sums_equal_unsharded(q, cfg_id, prec):
    cfg = wl.config(cfg_id)
    n_traj, steps, stride = 256 * 37 + 5, 200, cfg["out_stride"]
    n_out = steps // stride + 1
    m = q.Model(cfg["model"])

    def sums(first, count):
        run = q.Run(m, count, 3, prec, n_out, traj_id_offset=first)
        run.sample(cfg["init"])
        run.propagate(steps, cfg["dt"], stride)
        return run.sums()

    single = sums(0, n_traj)
    tile = q.shard_tile_walkers(m, prec)
    for world in (2, 4):
        parts = []
        for r in range(world):
            first, count = shard.shard_range(n_traj, world, r, tile)
            parts.append(sums(first, count) if count > 0 else np.zeros_like(single))
        assert np.array_equal(q.combine_shards(np.stack(parts)), single)
