"""Launch shapes of the FP32-bulk kernels (walkers per thread, blocks per SM,
output times per launch) change no bit of any result, and the autotuner picks
one of them."""
import copy

import numpy as np
import pytest

from paper_2608_14544_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch

    from paper_2608_14544_gb300 import build, qcl

    build.build()
    torch.cuda.set_device(0)
    return qcl


def _cases():
    c2 = wl.config(2)
    c3 = wl.config(3)
    d2 = copy.deepcopy(c2)
    d2["model"]["repr"] = "diabatic"
    c6 = copy.deepcopy(c3)
    c6["model"] = wl.random_lvc2(6, 3, 0.1)
    c6["init"] = wl.sb_init(c6["model"], beta=2.0)
    c4 = wl.config(4)
    c80 = copy.deepcopy(c3)
    c80["model"] = wl.random_lvc2(80, 5, 0.1)
    c80["init"] = wl.sb_init(c80["model"], beta=2.0)
    c4d = copy.deepcopy(c4)
    c4d["model"]["repr"] = "diabatic"
    lvc40 = wl.lvc4_config(2, 40)
    lvc40d = copy.deepcopy(lvc40)
    lvc40d["model"]["repr"] = "diabatic"
    return [("sb3", c2), ("vib3", c3), ("sb3-diabatic", d2), ("lvc2-6mode", c6),
            ("lvc4", wl.lvc4_config(2)), ("sb100-split", c4), ("lvc2-80mode-split", c80),
            ("sb100-diabatic-split", c4d), ("lvc4-40mode-in-memory", lvc40),
            ("lvc4-40mode-diabatic-in-memory", lvc40d)]


@pytest.mark.parametrize("name,cfg", _cases())
def test_every_launch_shape_gives_the_same_bits(q, name, cfg):
    # 586 tiles: more than the resident block slots at every shape, so that
    # walkers-per-thread 2 is launched as asked (smaller ensembles run 1)
    n, steps, stride = 150_001, 120, 10
    outs = []
    for wpt, bps, opl in ((1, 0, 0), (2, 0, 0), (1, 1, 8), (2, 1, 16), (0, 2, 1), (0, 0, 3)):
        m = q.Model(cfg["model"])
        m.set_launch_shape(wpt, bps, opl)
        run = q.Run(m, n, 6, q.PREC_FP32_BULK, steps // stride + 1)
        run.sample(cfg["init"])
        run.propagate(55, cfg["dt"], stride)
        run.propagate(steps - 55, cfg["dt"], stride)
        outs.append((run.sums(), run.state()))
        assert run.status()["flags"] == 0
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0]), name
        for k in st:
            assert np.array_equal(st[k], outs[0][1][k]), (name, k)


def test_autotune_picks_a_measured_shape(q):
    cfg = wl.config(2)
    m = q.Model(cfg["model"])
    best = m.autotune(cfg["dt"], cfg["out_stride"], probe_walkers=1 << 19, n_steps=80)
    assert best["walkers_per_thread"] in (1, 2)
    assert best["blocks_per_sm"] >= 1
    assert best["outputs_per_launch"] in (8, 16, 32)
    assert best["walker_steps_per_s"] > 1e9
    assert m.launch_shape() == best
    # the model keeps solving with the tuned shape, same bits as the default
    res = []
    for mm in (m, q.Model(cfg["model"])):
        run = q.Run(mm, 50_000, 1, q.PREC_FP32_BULK, 11)
        run.sample(cfg["init"])
        run.propagate(100, cfg["dt"], 10)
        res.append(run.sums())
    assert np.array_equal(res[0], res[1])


def test_launch_shape_range_is_checked(q):
    m = q.Model(wl.config(1)["model"])
    for bad in ((3, 0, 0), (0, -1, 0), (0, 0, 33), (0, 0, -1)):
        with pytest.raises(q.QclError) as e:
            m.set_launch_shape(*bad)
        assert e.value.status == 1


def test_fma_microbenchmarks_are_plausible(q):
    import torch

    props = torch.cuda.get_device_properties(0)
    fp32 = q.measure_peak(0)
    fp64 = q.measure_peak(1)
    # FP32: 128 lanes x 2 flop per SM-cycle at 1-2.1 GHz
    per_sm_cycle = fp32 / props.multi_processor_count / 2.1e9
    assert 0.3 * 256 < per_sm_cycle < 1.05 * 256, per_sm_cycle
    assert 0 < fp64 < fp32
