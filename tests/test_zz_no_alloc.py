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
    return rows.cpu().numpy()


def test_noalloc_rows_match_propagate_on_two_calls(q):
    # two calls in a row: a large ensemble (several launches per call, since
    # fewer output times fit the static scratch) and then a small ragged one,
    # so the second call runs over the first one's leftovers
    for cfg_id, n, splits, seed in ((2, 4_000_000, (130, 270), 5), (3, 3001, (200,), 9)):
        cfg = wl.config(cfg_id)
        stride = cfg["out_stride"]
        ref, _ = _reference_rows(q, cfg, n, seed, splits, stride)
        got = _noalloc_rows(q, cfg, n, seed, splits, stride)
        assert np.all(np.isfinite(got))
        scale = np.sqrt(n * np.abs(ref[:, 16:])) + 1e-300
        assert np.all(np.abs(got[:, :16] - ref[:, :16]) <= 1e-12 * scale)
        assert np.allclose(got[:, 16:], ref[:, 16:], rtol=1e-12, atol=0)


def test_noalloc_rejects_walker_counts_beyond_the_static_scratch(q):
    cfg = wl.config(2)
    m = q.Model(cfg["model"])
    ens = q.ens_desc(200_000_000, 0, q.PREC_FP32_BULK)
    import ctypes as C

    st = q.load().qcl_propagate_noalloc(m.handle, C.byref(ens), None, 0, 0, 10, 0.01, 10, None,
                                        0, 2, None)
    assert st == 2  # QCL_ERR_UNSUPPORTED
    assert "static scratch" in q.last_error()
    fp64 = q.ens_desc(1000, 0, q.PREC_FP64)
    st = q.load().qcl_propagate_noalloc(m.handle, C.byref(fp64), None, 0, 0, 10, 0.01, 10, None,
                                        0, 2, None)
    assert st == 2
