"""Models with more than two electronic states (Jacobi decomposition carried
along each trajectory with parallel-transport gauge): FP64 path per trajectory
against the oracle, FP32-bulk ensemble against the FP64 path and the oracle,
bitwise chunk invariance."""
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


def _model3():
    rng = np.random.default_rng(5)
    n = 4
    omega = rng.uniform(0.6, 1.5, size=n)
    E = np.diag([0.0, 0.4, 0.9]) + 0.05 * (np.ones((3, 3)) - np.eye(3))
    K = np.zeros((n, 3, 3))
    for j in range(n):
        a = rng.normal(size=(3, 3)) * 0.15
        K[j] = 0.5 * (a + a.T)
    return wl._model(E, K, np.ones(n), omega, name="lvc3")


def _cases():
    m4 = wl.random_lvc4(11)
    return [("lvc4", m4, wl.sb_init(m4, beta=2.0), 0.01),
            ("lvc3", _model3(), wl.sb_init(_model3(), beta=3.0), 0.01)]


def _run(q, model, init, n, prec, seed, n_out, splits=(), dt=0.01, stride=10, cap=0):
    q.set_option(q.OPT_GRID_CAP, cap)
    m = q.Model(model)
    run = q.Run(m, n, seed, prec, n_out)
    run.sample(init)
    for k in splits:
        run.propagate(k, dt, stride)
    q.set_option(q.OPT_GRID_CAP, 0)
    return run


def _to_oracle(om, st):
    s = oracle.State(om, len(st["m"]))
    s.R[:] = st["R"]
    s.P[:] = st["P"]
    s.m[:] = st["m"]
    s.phi[:] = st["phi"]
    s.alpha[:] = st["alpha"]
    s.beta[:] = st["beta"]
    s.U[:] = st["U"]
    return s


@pytest.mark.parametrize("case", [0, 1])
def test_nstate_fp64_sample_matches_oracle(q, case):
    name, model, init, dt = _cases()[case]
    run = _run(q, model, init, 777, q.PREC_FP64, 4, 2)
    st = run.state()
    om = oracle.OracleModel(model)
    ref = oracle.sample(om, oracle.OracleInit(om, init), 4, 0, 777)
    assert np.allclose(st["R"], ref.R, rtol=1e-13, atol=1e-14)
    assert np.array_equal(st["alpha"], ref.alpha) and np.array_equal(st["beta"], ref.beta)
    assert np.allclose(st["m"], ref.m, rtol=1e-11)
    assert np.allclose(st["U"], ref.U, atol=1e-12)


@pytest.mark.parametrize("case", [0, 1])
def test_nstate_fp64_per_trajectory_parity(q, case):
    """R, P, phi, U and the weight per trajectory to 1e-12 over 50-step segments,
    each restarted from the GPU's own checkpoint; identical decisions."""
    name, model, init, dt = _cases()[case]
    n, seg, steps = 2000, 50, 300
    run = _run(q, model, init, n, q.PREC_FP64, 6, steps // 10 + 1)
    om = oracle.OracleModel(model)
    worst = {}
    flips = 0
    for s0 in range(0, steps, seg):
        ref = _to_oracle(om, run.state())
        oracle.advance(om, ref, 6, 0, s0, seg, dt)
        run.propagate(seg, dt, 10)
        g = run.state()
        same = (g["alpha"] == ref.alpha) & (g["beta"] == ref.beta)
        flips += int((~same).sum())
        for key, r in (("R", ref.R), ("P", ref.P), ("phi", ref.phi)):
            err = np.abs(g[key][same] - r[same]) / np.maximum(np.abs(r[same]), 1.0)
            worst[key] = max(worst.get(key, 0.0), float(err.max()))
        worst["U"] = max(worst.get("U", 0.0), float(np.abs(g["U"][same] - ref.U[same]).max()))
        merr = np.abs(g["m"][same] - ref.m[same]) / np.abs(ref.m[same])
        worst["m"] = max(worst.get("m", 0.0), float(merr.max()))
    assert flips == 0
    assert max(worst.values()) < 1e-12, worst


@pytest.mark.parametrize("case", [0, 1])
def test_nstate_fp32_matches_fp64_and_oracle(q, case):
    name, model, init, dt = _cases()[case]
    steps, stride = 400, 10
    n_out = steps // stride + 1
    a = _run(q, model, init, 200_000, q.PREC_FP64, 8, n_out, (steps,)).observables()
    rb = _run(q, model, init, 200_000, q.PREC_FP32_BULK, 8, n_out, (steps,))
    b = rb.observables()
    assert rb.status()["flags"] == 0
    nq = 4 * model["n_states"] ** 2
    se = np.sqrt(a[:, nq:2 * nq] ** 2 + b[:, nq:2 * nq] ** 2)
    diff = np.abs(a[:, :nq] - b[:, :nq])
    assert np.all(diff <= 3 * se + 1e-9), (diff / (se + 1e-300)).max()
    resolved = se.max(axis=1) < 1e-2
    assert resolved.sum() >= 5
    assert diff[resolved].max() < 1e-3
    # ensemble of 3000 walkers against the oracle
    n = 3000
    c = _run(q, model, init, n, q.PREC_FP32_BULK, 9, n_out, (steps,)).observables()
    om = oracle.OracleModel(model)
    ref, _ = oracle.run(om, oracle.OracleInit(om, init), 9, 0, n, dt, steps, stride)
    mean, se_o = oracle.finalize(ref, n)
    d = np.abs(c[:, :nq] - mean)
    assert np.all(d <= 3 * se_o + 1e-9), (d / (se_o + 1e-300)).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_nstate_chunking_and_launch_shape_bitwise(q, prec):
    name, model, init, dt = _cases()[0]
    outs = []
    for splits, cap in (((200,), 0), ((70, 130), 0), ((200,), 3)):
        r = _run(q, model, init, 9000, prec, 2, 21, splits, cap=cap)
        outs.append((r.sums(), r.state()))
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0])
        for k in st:
            assert np.array_equal(st[k], outs[0][1][k]), k
