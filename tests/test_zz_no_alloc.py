"""qcl_propagate_noalloc: FP32-bulk propagation for callers that cannot
allocate device memory while they propagate (a service that reserved its
device memory up front, a plug-in handed fixed buffers).  Its scratch is a
static device array inside the library, so its output rows must equal those
of qcl_propagate, which keeps the same scratch in the caller's observation
buffer.  This file is collected last on purpose; it must pass alone in a fresh
process and after the other tests.
"""
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


def _reference_rows(q, cfg, n, seed, splits, stride):
    m = q.Model(cfg["model"])
    n_out = sum(splits) // stride + 1
    run = q.Run(m, n, seed, q.PREC_FP32_BULK, n_out)
    run.sample(cfg["init"])
    for k in splits:
        run.propagate(k, cfg["dt"], stride)
    return run.sums(), run.state()


def _noalloc_rows(q, cfg, n, seed, splits, stride):
    import torch

    m = q.Model(cfg["model"])
    n_out = sum(splits) // stride + 1
    ens = q.ens_desc(n, seed, q.PREC_FP32_BULK)
    ens_buf = q.device_buffer(q.ensemble_bytes(m, ens))
    rows = torch.full((n_out, 8 * m.ns * m.ns), float("nan"), dtype=torch.float64,
                      device="cuda")
    q.sample_initial(m, ens, cfg["init"], ens_buf)
    step = 0
    for k in splits:  # consecutive calls on the same ensemble share the static scratch
        q.propagate_noalloc(m, ens, ens_buf, step, k, cfg["dt"], stride, rows, n_out)
        step += k
    torch.cuda.synchronize()
    st = q.ensemble_status(m, ens, ens_buf)
    assert st["step"] == step and st["flags"] == 0, st
    view = q.Run.__new__(q.Run)  # the state reader of a Run over this buffer
    view.model, view.ens, view.ens_buf = m, ens, ens_buf
    return rows.cpu().numpy(), view.state()


def test_noalloc_rows_match_propagate_on_two_calls(q):
    """The same bits as qcl_propagate, rows and walker states, on two calls in
    a row per case.  The cases cover: several launches per call (fewer output
    times fit the static scratch than the call spans), a small ragged ensemble
    that runs over the previous case's leftovers, a many-mode model (its
    walkers' modes split over four warps, 64-walker tiles) with so many walkers
    that only one output time fits per launch (the output at t = 0 then gets a
    launch of its own), and the same kernel with a handful of walkers."""
    cases = ((2, 4_000_000, (130, 270), 5), (3, 3001, (200,), 9),
             (4, 6_000_000, (40, 60), 2), (4, 2001, (37, 23), 4))
    for cfg_id, n, splits, seed in cases:
        cfg = wl.config(cfg_id)
        stride = cfg["out_stride"]
        ref, ref_state = _reference_rows(q, cfg, n, seed, splits, stride)
        got, got_state = _noalloc_rows(q, cfg, n, seed, splits, stride)
        assert np.all(np.isfinite(got)), cfg_id
        assert np.array_equal(got, ref), (cfg_id, n)
        for k in ref_state:
            assert np.array_equal(got_state[k], ref_state[k]), (cfg_id, n, k)


def test_noalloc_rejects_walker_counts_beyond_the_static_scratch(q):
    """Past the static array's capacity (about 33 million walkers of a
    3-mode model) the call fails with QCL_ERR_UNSUPPORTED and says so, after
    the argument checks it shares with qcl_propagate; an FP64 ensemble is
    rejected the same way."""
    import torch

    cfg = wl.config(2)
    m = q.Model(cfg["model"])
    n_out = 2
    rows = torch.zeros((n_out, 8 * m.ns * m.ns), dtype=torch.float64, device="cuda")
    ens = q.ens_desc(40_000_000, 0, q.PREC_FP32_BULK)
    buf = q.device_buffer(q.ensemble_bytes(m, ens))
    with pytest.raises(q.QclError) as e:
        q.propagate_noalloc(m, ens, buf, 0, 10, cfg["dt"], 10, rows, n_out)
    assert e.value.status == 2 and "static scratch" in q.last_error()
    # an argument error is reported first, with qcl_propagate's code
    with pytest.raises(q.QclError) as e:
        q.propagate_noalloc(m, ens, buf, 0, 10, -1.0, 10, rows, n_out)
    assert e.value.status == 1
    del buf
    fp64 = q.ens_desc(1000, 0, q.PREC_FP64)
    buf64 = q.device_buffer(q.ensemble_bytes(m, fp64))
    with pytest.raises(q.QclError) as e:
        q.propagate_noalloc(m, fp64, buf64, 0, 10, cfg["dt"], 10, rows, n_out)
    assert e.value.status == 2 and "FP32-bulk" in q.last_error()


def test_noalloc_diabatic_many_mode_matches_propagate(q):
    """The diabatic representation of the 100-mode model (the split kernel's
    diabatic form, 64-walker tiles) through the no-allocation call: the same
    rows and walker states as qcl_propagate."""
    import copy

    cfg = copy.deepcopy(wl.config(4))
    cfg["model"]["repr"] = "diabatic"
    stride = cfg["out_stride"]
    ref, ref_state = _reference_rows(q, cfg, 30_001, 7, (60, 40), stride)
    got, got_state = _noalloc_rows(q, cfg, 30_001, 7, (60, 40), stride)
    assert np.array_equal(got, ref)
    for k in ref_state:
        assert np.array_equal(got_state[k], ref_state[k]), k
