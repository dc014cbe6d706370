"""Many-mode two-state models (33..256 modes) in the diabatic representation on
the FP32-bulk path (the split kernel's diabatic form: a walker's modes over 2
or 4 warps, one exchange of a(R), b(R) per step): against the FP64 path and the
oracle on matched walkers, per walker against the FP64 path over segments
restarted from its checkpoint, bitwise invariance under chunking, launch shape
and serving."""
import numpy as np
import pytest

import oracle
from paper_2608_14544_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch

    from paper_2608_14544_gb300 import build, qcl

    build.build()
    oracle.build()
    torch.cuda.set_device(0)
    return qcl


def _case(n_modes, kind):
    if kind == "sb":
        w, c = wl.ohmic_modes(n_modes, 0.25, 5.0)
        model = wl.spin_boson(1.0, 1.0, w, c)
        init = wl.sb_init(model, beta=1.0)
        dt = 0.005
    else:
        model = wl.random_lvc2(n_modes, seed=n_modes, scale=0.1)
        init = wl.sb_init(model, beta=2.0)
        dt = 0.01
    model["repr"] = "diabatic"
    return model, init, dt


def _run(q, model, init, n, prec, steps, stride, dt, seed, splits=None, cap=0):
    q.set_option(q.OPT_GRID_CAP, cap)
    try:
        run = q.Run(q.Model(model), n, seed, prec, steps // stride + 1)
        run.sample(init)
        for k in (splits or (steps,)):
            run.propagate(k, dt, stride)
    finally:
        q.set_option(q.OPT_GRID_CAP, 0)
    return run


# (33, 65 and 129 modes: the first model of each split range -- two roles of 32,
# four of 32, four of 64 with shared-memory coefficients)
@pytest.mark.parametrize("n_modes,kind", [(40, "sb"), (100, "sb"), (200, "sb"), (33, "lvc"),
                                          (65, "lvc"), (129, "lvc")])
def test_manymode_dia_fp32_matches_fp64(q, n_modes, kind):
    model, init, dt = _case(n_modes, kind)
    steps, stride, n = 300, 10, 200_000
    a = _run(q, model, init, n, q.PREC_FP64, steps, stride, dt, 3).observables()
    rb = _run(q, model, init, n, q.PREC_FP32_BULK, steps, stride, dt, 3)
    assert rb.status()["flags"] == 0
    b = rb.observables()
    assert q.shard_tile_walkers(q.Model(model), q.PREC_FP32_BULK) == (128 if n_modes <= 64 else 64)
    se = np.sqrt(a[:, 16:32] ** 2 + b[:, 16:32] ** 2)
    diff = np.abs(a[:, :16] - b[:, :16])
    assert np.all(np.isfinite(b[:, :32]))
    assert np.all(diff <= 3.5 * se + 1e-9), (diff / (se + 1e-300)).max()
    assert diff[0].max() < 1e-5  # the same sample
    resolved = se.max(axis=1) < 1e-2
    assert resolved.sum() >= 4
    assert diff[resolved].max() < 1e-3
    # the populations move in the resolved window
    assert np.abs(a[resolved, 14] - a[0, 14]).max() > 1e-3


def test_manymode_dia_fp32_matches_oracle(q):
    model, init, dt = _case(100, "sb")
    n, steps, stride = 1500, 400, 20
    obs = _run(q, model, init, n, q.PREC_FP32_BULK, steps, stride, dt, 7).observables()
    om = oracle.OracleModel(model)
    ref, _ = oracle.run(om, oracle.OracleInit(om, init), 7, 0, n, dt, steps, stride)
    mean, se = oracle.finalize(ref, n)
    diff = np.abs(obs[:, :16] - mean)
    assert np.all(diff <= 3 * se + 1e-9), (diff / (se + 1e-300)).max()
    ok = se < 1e-2
    if ok.any():
        assert diff[ok].max() < 1e-3


def _to_fp32(ck):
    m = np.asarray(ck["m"], dtype=np.float64)
    _, e2 = np.frexp(m)
    ex = np.where(m != 0, e2 - 1, 0).astype(np.int32)
    mant = np.ldexp(m, -ex)
    mhi = mant.astype(np.float32)
    mlo = (mant - mhi.astype(np.float64)).astype(np.float32)
    phi = np.asarray(ck["phi"], dtype=np.float64)
    phi_hi = phi.astype(np.float32)
    phi_lo = (phi - phi_hi.astype(np.float64)).astype(np.float32)
    return {"R": ck["R"].astype(np.float32), "P": ck["P"].astype(np.float32), "m": mhi,
            "m_lo": mlo, "m_exp": ex, "phi": phi_hi, "phi_lo": phi_lo,
            "alpha": ck["alpha"], "beta": ck["beta"], "q": ck["q"]}


def _as_fp64(st):
    return {"R": st["R"].astype(np.float64), "P": st["P"].astype(np.float64),
            "m": (st["m"].astype(np.float64) + st["m_lo"].astype(np.float64))
            * np.ldexp(1.0, st["m_exp"]),
            "phi": st["phi"].astype(np.float64) + st["phi_lo"].astype(np.float64),
            "alpha": st["alpha"], "beta": st["beta"], "q": st["q"]}


@pytest.mark.parametrize("n_modes,kind", [(100, "sb"), (65, "lvc")])
def test_manymode_dia_per_walker_vs_fp64(q, n_modes, kind):
    """Over 40-step segments from the FP64 path's checkpoint: at least 99.9 % of
    the walkers take the same decisions; for those, R, P and phase within 1e-5
    relative (99.9 %, all within 1e-3) and the weight within 1e-5 for 99 % (the
    rest carry a 24-bit threshold that the precisions round to neighbouring
    integers: within 1e-3)."""
    model, init, dt = _case(n_modes, kind)
    n, seed, seg, stride = 60_000, 5, 40, 10
    starts = [0, 200]
    n_out = (starts[-1] + seg) // stride + 1
    m = q.Model(model)
    r64 = q.Run(m, n, seed, q.PREC_FP64, n_out)
    r64.sample(init)
    r32 = q.Run(m, n, seed, q.PREC_FP32_BULK, n_out)
    tol = 1e-5
    for s0 in starts:
        if r64.step < s0:
            r64.propagate(s0 - r64.step, dt, stride)
        r32.load_state(_to_fp32(r64.state()), s0)
        matched = np.ones(n, dtype=bool)
        for _ in range(seg // 10):
            r64.propagate(10, dt, stride)
            r32.propagate(10, dt, stride)
            g, f = r64.state(), r32.state()
            matched &= ((f["alpha"] == g["alpha"]) & (f["beta"] == g["beta"])
                        & (f["q"] == g["q"]))
        assert r32.status()["flags"] == 0
        assert matched.mean() > 0.999, matched.mean()
        f = _as_fp64(r32.state())
        for key in ("R", "P", "phi"):
            if key == "phi":
                err = np.abs(f[key] - g[key]) / np.maximum(np.abs(g[key]), 1.0)
            else:
                scale = np.maximum(np.abs(g[key]), g[key].std(axis=0, keepdims=True))
                err = (np.abs(f[key] - g[key]) / scale).max(axis=1)
            assert (err[matched] > tol).mean() < 1e-3, (key, s0)
            assert err[matched].max() < 1e-3, (key, s0, err[matched].max())
        err_m = (np.abs(f["m"] - g["m"]) / np.abs(g["m"]))[matched]
        assert (err_m > tol).mean() < 0.01, (s0, (err_m > tol).mean())
        assert err_m.max() < 1e-3, (s0, err_m.max())
        moved = (g["alpha"] != 0) | (g["beta"] != 0)
        assert moved.any()


@pytest.mark.parametrize("n_modes", [64, 100, 200])
def test_manymode_dia_chunking_and_launch_shape_bitwise(q, n_modes):
    model, init, dt = _case(n_modes, "lvc" if n_modes != 200 else "sb")
    outs = []
    for splits, cap in (((200,), 0), ((70, 130), 0), ((200,), 5)):
        r = _run(q, model, init, 20_000, q.PREC_FP32_BULK, 200, 10, dt, 2, splits, cap)
        outs.append((r.sums(), r.state()))
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0])
        for k in st:
            assert np.array_equal(st[k], outs[0][1][k]), k


def test_served_manymode_dia_equals_single_solve(q):
    model, init, dt = _case(100, "sb")
    n, steps, stride = 40_000, 200, 10
    single = _run(q, model, init, n, q.PREC_FP32_BULK, steps, stride, dt, 21).observables()
    srv = q.Server(1 << 30, quantum_steps=70)
    rid = srv.submit(dict(model=model, init=init, n_traj=n, seed=21, n_steps=steps, dt=dt,
                          out_stride=stride))
    st, obs = srv.wait(rid)
    srv.close()
    assert st == q.REQ_DONE
    assert np.array_equal(obs, single)
