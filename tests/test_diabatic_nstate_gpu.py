"""The diabatic representation for models with more than two states: the
walkers' index pairs in the R-independent basis of W, the coupling as the
off-diagonal potential (events a -> g with amplitude -i W_ga dt / hbar and
b -> g with +i W_bg dt / hbar, weights carried with a quarter-turn count).
FP64 path per trajectory against the oracle, FP32-bulk ensemble against the
FP64 path and against the oracle on the same walkers, bitwise chunk and launch
shape invariance, served equal to the single solve."""
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
    """Three states with off-diagonal couplings in E and in every K_j."""
    rng = np.random.default_rng(7)
    n = 4
    omega = rng.uniform(0.6, 1.5, size=n)
    E = np.diag([0.0, 0.3, 0.7]) + 0.08 * (np.ones((3, 3)) - np.eye(3))
    K = np.zeros((n, 3, 3))
    for j in range(n):
        a = rng.normal(size=(3, 3)) * 0.15
        K[j] = 0.5 * (a + a.T)
    m = wl._model(E, K, np.ones(n), omega, name="lvc3-dia")
    m["repr"] = "diabatic"
    return m


def _cases():
    m4 = wl.random_lvc4(11)
    m4["repr"] = "diabatic"
    m3 = _model3()
    return [("lvc4-dia", m4, wl.sb_init(m4, beta=2.0), 0.01),
            ("lvc3-dia", m3, wl.sb_init(m3, beta=3.0), 0.01)]


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
    s.q[:] = st["q"]
    if "U" in st:
        s.U[:] = st["U"]
    return s


@pytest.mark.parametrize("case", [0, 1])
def test_diabatic_nstate_fp64_sample_matches_oracle(q, case):
    name, model, init, dt = _cases()[case]
    st = _run(q, model, init, 777, q.PREC_FP64, 4, 2).state()
    om = oracle.OracleModel(model)
    ref = oracle.sample(om, oracle.OracleInit(om, init), 4, 0, 777)
    assert np.allclose(st["R"], ref.R, rtol=1e-13, atol=1e-14)
    assert np.array_equal(st["alpha"], ref.alpha) and np.array_equal(st["beta"], ref.beta)
    assert np.all(st["q"] == 0)
    assert np.allclose(st["m"], ref.m, rtol=1e-11)
    # pairs drawn from rho_el0 itself: the diabatic |0><0| start puts every walker at (0, 0)
    assert np.all(st["alpha"] == 0) and np.all(st["beta"] == 0)


@pytest.mark.parametrize("case", [0, 1])
def test_diabatic_nstate_fp64_per_trajectory_parity(q, case):
    """R, P, phi and the weight per trajectory to 1e-12 over 50-step segments,
    each restarted from the GPU's own checkpoint; identical pairs and quarter
    turns; transitions do fire."""
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
        same = (g["alpha"] == ref.alpha) & (g["beta"] == ref.beta) & (g["q"] == ref.q)
        flips += int((~same).sum())
        for key, r in (("R", ref.R), ("P", ref.P), ("phi", ref.phi)):
            err = np.abs(g[key][same] - r[same]) / np.maximum(np.abs(r[same]), 1.0)
            worst[key] = max(worst.get(key, 0.0), float(err.max()))
        merr = np.abs(g["m"][same] - ref.m[same]) / np.abs(ref.m[same])
        worst["m"] = max(worst.get("m", 0.0), float(merr.max()))
    assert flips == 0
    assert max(worst.values()) < 1e-12, worst
    g = run.state()
    moved = (g["alpha"] != 0) | (g["beta"] != 0)
    assert moved.mean() > 0.05, moved.mean()
    assert np.any(g["q"] != 0)


@pytest.mark.parametrize("case", [0, 1])
def test_diabatic_nstate_fp64_observables_match_oracle(q, case):
    """The FP64 path's observable sums (pairwise per tile, then the fixed tile
    fold) against the oracle's (one pairwise tree) on the same walkers, to
    rounding; the adiabatic block rotated by the eigenvectors at each walker's
    R with the oracle's sign convention."""
    name, model, init, dt = _cases()[case]
    n, steps, stride = 3000, 120, 10
    g = _run(q, model, init, n, q.PREC_FP64, 12, steps // stride + 1, (steps,)).observables()
    om = oracle.OracleModel(model)
    ref, _ = oracle.run(om, oracle.OracleInit(om, init), 12, 0, n, dt, steps, stride)
    mean, se = oracle.finalize(ref, n)
    nq = 4 * model["n_states"] ** 2
    assert np.allclose(g[:, :nq], mean, rtol=1e-9, atol=1e-11), np.abs(g[:, :nq] - mean).max()
    assert np.allclose(g[:, nq:2 * nq], se, rtol=1e-7, atol=1e-11)


@pytest.mark.parametrize("case", [0, 1])
def test_diabatic_nstate_fp32_matches_fp64_and_oracle(q, case):
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
    # the same walkers (seed, ids, Philox streams) in the oracle: 3000 walkers
    n = 3000
    c = _run(q, model, init, n, q.PREC_FP32_BULK, 9, n_out, (steps,)).observables()
    om = oracle.OracleModel(model)
    ref, _ = oracle.run(om, oracle.OracleInit(om, init), 9, 0, n, dt, steps, stride)
    mean, se_o = oracle.finalize(ref, n)
    d = np.abs(c[:, :nq] - mean)
    assert np.all(d <= 3 * se_o + 1e-9), (d / (se_o + 1e-300)).max()
    ok = se_o.max(axis=1) < 1e-2
    assert d[ok].max() < 1e-3


@pytest.mark.parametrize("prec", [0, 1])
def test_diabatic_nstate_chunking_and_launch_shape_bitwise(q, prec):
    name, model, init, dt = _cases()[0]
    outs = []
    for splits, cap in (((200,), 0), ((70, 130), 0), ((200,), 3)):
        r = _run(q, model, init, 9000, prec, 2, 21, splits, cap=cap)
        outs.append((r.sums(), r.state()))
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0])
        for k in st:
            assert np.array_equal(st[k], outs[0][1][k]), k


def test_diabatic_nstate_served_equals_single_solve(q):
    name, model, init, dt = _cases()[1]
    n, steps, stride = 50_000, 200, 10
    single = _run(q, model, init, n, q.PREC_FP32_BULK, 21, steps // stride + 1,
                  (steps,)).observables()
    srv = q.Server(1 << 30, quantum_steps=70)
    rid = srv.submit(dict(model=model, init=init, n_traj=n, seed=21, n_steps=steps, dt=dt,
                          out_stride=stride))
    st, obs = srv.wait(rid)
    srv.close()
    assert st == q.REQ_DONE
    assert np.array_equal(obs, single)


def test_diabatic_nstate_frozen_nuclei_populations_are_exact_on_average(q):
    """K = 0 (frozen nuclei): the diabatic estimator's expectation obeys the
    linear recursion of the oracle's pins; the FP32-bulk ensemble tracks the
    exact diagonal-phase / first-order-transfer recursion within its standard
    error at every output."""
    E = np.array([[0.3, 0.25, 0.1], [0.25, -0.2, 0.15], [0.1, 0.15, 0.05]])
    model = wl._model(E, np.zeros((1, 3, 3)), np.ones(1), np.ones(1), name="frozen3")
    model["repr"] = "diabatic"
    rho0 = np.array([[0.6, 0.2, 0.1], [0.2, 0.3, 0.05], [0.1, 0.05, 0.1]])
    init = {"rho_el0": rho0, "R0": np.zeros(1), "P0": np.zeros(1), "beta": np.inf, "wigner": 1}
    dt, steps, stride, n = 0.05, 80, 10, 400_000
    got = _run(q, model, init, n, q.PREC_FP32_BULK, 17, steps // stride + 1, (steps,), dt=dt,
               stride=stride).observables()
    d = np.diag(E)
    Phi = np.exp(-1j * (d[:, None] - d[None, :]) * dt)
    Cm = (E - np.diag(d)) * dt
    rho = rho0.astype(complex)
    want = [rho.copy()]
    for _ in range(steps):
        D = Phi * rho
        rho = D - 1j * (Cm @ D) + 1j * (D @ Cm)
        want.append(rho.copy())
    want = np.array(want)[::stride].reshape(-1, 9)
    ns = 3
    nq = 4 * ns * ns
    g = got[:, 0:2 * ns * ns:2] + 1j * got[:, 1:2 * ns * ns:2]
    se = got[:, nq:nq + 2 * ns * ns:2] + 1j * got[:, nq + 1:nq + 2 * ns * ns:2]
    z_re = np.abs(g.real - want.real) / np.maximum(se.real, 1e-15)
    z_im = np.abs(g.imag - want.imag) / np.maximum(se.imag, 1e-15)
    assert np.all((z_re < 4.5) | (np.abs(g.real - want.real) < 1e-6)), z_re.max()
    assert np.all((z_im < 4.5) | (np.abs(g.imag - want.imag) < 1e-6)), z_im.max()
    assert np.abs(want - want[0]).max() > 0.05  # the populations moved
