"""Trajectory spawning for models with more than two states (FP64, both
representations) against the oracle: per-walker parity (same walker list,
ids and families; R, P, phi, m to 1e-12) over segments restarted from the
GPU's own checkpoint, family-summed observables, chunk invariance, and the
capacity-overflow flag."""
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


def _model3(rep):
    rng = np.random.default_rng(13)
    n = 3
    omega = rng.uniform(0.6, 1.5, size=n)
    E = np.diag([0.0, 0.4, 0.8]) + 0.05 * (np.ones((3, 3)) - np.eye(3))
    K = np.zeros((n, 3, 3))
    for j in range(n):
        a = rng.normal(size=(3, 3)) * 0.12
        K[j] = 0.5 * (a + a.T)
    m = wl._model(E, K, np.ones(n), omega, name=f"lvc3-{rep}")
    m["repr"] = rep
    return m


def _case(rep):
    m = _model3(rep)
    # (the population grows about 5x (adiabatic) and 2x (diabatic) in 160 steps)
    return m, wl.sb_init(m, beta=3.0), 0.01


def _oracle_from_gpu(om, st, n0, cap):
    s = oracle.SpawnState(om, n0, cap)
    k = len(st["m"])
    s.n_live = k
    for key in ("R", "P", "m", "phi", "alpha", "beta", "q", "id", "family"):
        getattr(s, key)[:k] = st[key]
    if "U" in st:
        s.U[:k] = st["U"]
    return s


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_spawn_nstate_per_walker_parity(q, rep):
    model, init, dt = _case(rep)
    n0, steps, seg, stride = 500, 160, 40, 10
    cap = 80 * n0
    m = q.Model(model)
    run = q.SpawnRun(m, n0, cap, 5, steps // stride + 1, traj_id_offset=100)
    run.sample(init)
    om = oracle.OracleModel(model)
    ref0 = oracle.spawn_sample(om, oracle.OracleInit(om, init), 5, 100, n0, cap)
    st = run.state()
    for key in ("alpha", "beta", "q", "id", "family"):
        assert np.array_equal(st[key], ref0.live()[key]), key
    if rep == "adiabatic":
        assert np.allclose(st["U"], ref0.U[:n0], atol=1e-12)
    worst = {}
    for s0 in range(0, steps, seg):
        ck = run.state()
        ref = _oracle_from_gpu(om, ck, n0, cap)
        assert oracle.spawn_advance(om, ref, 5, s0, seg, dt) == 0
        run.propagate(seg, dt, stride)
        g = run.state()
        r = ref.live()
        assert len(g["m"]) == len(r["m"]), (s0, len(g["m"]), len(r["m"]))
        for key in ("alpha", "beta", "q", "id", "family"):
            assert np.array_equal(g[key], r[key]), (s0, key)
        for key in ("R", "P", "phi", "m"):
            den = np.abs(r[key]) + 1e-300 if key == "m" else np.maximum(np.abs(r[key]), 1.0)
            worst[key] = max(worst.get(key, 0.0), float((np.abs(g[key] - r[key]) / den).max()))
        if rep == "adiabatic":
            k = len(g["m"])
            worst["U"] = max(worst.get("U", 0.0), float(np.abs(g["U"] - ref.U[:k]).max()))
    assert max(worst.values()) < 1e-12, worst
    assert run.n_live() > 1.2 * n0  # children were spawned
    assert run.status()["flags"] & q.FLAG_SPAWN_OVERFLOW == 0
    if rep == "diabatic":
        assert np.any(run.state()["q"] != 0)


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_spawn_nstate_observables_match_oracle(q, rep):
    model, init, dt = _case(rep)
    n0, steps, stride, cap = 800, 120, 10, 200_000
    m = q.Model(model)
    run = q.SpawnRun(m, n0, cap, 3, steps // stride + 1)
    run.sample(init)
    run.propagate(steps, dt, stride)
    sums = run.sums()
    om = oracle.OracleModel(model)
    ref, n_live = oracle.run_spawn(om, oracle.OracleInit(om, init), 3, 0, n0, cap, dt, steps,
                                   stride)
    nq = 4 * model["n_states"] ** 2
    scale = np.sqrt(n0 * np.abs(ref[:, nq:])) + 1e-300
    err = np.abs(sums[:, :nq] - ref[:, :nq]) / scale
    assert err.max() < 1e-10, err.max()
    assert np.allclose(sums[:, nq:], ref[:, nq:], rtol=1e-9, atol=1e-12)
    assert run.n_live() == n_live[-1]
    obs = run.observables()
    assert np.allclose(obs[:, 2 * nq + 2], n0)  # means and errors are over the n0 families


def test_spawn_nstate_chunking_is_bitwise_invisible(q):
    model, init, dt = _case("adiabatic")
    n0, cap = 600, 120_000
    outs = []
    for split in ((100,), (30, 70), (1, 49, 50)):
        m = q.Model(model)
        run = q.SpawnRun(m, n0, cap, 4, 100 // 10 + 1)
        run.sample(init)
        for k in split:
            run.propagate(k, dt, 10)
        outs.append((run.sums(), run.state()))
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0])
        for key in st:
            assert np.array_equal(st[key], outs[0][1][key]), key


def test_spawn_nstate_overflow_sets_flag(q):
    model, init, dt = _case("diabatic")
    n0 = 300
    m = q.Model(model)
    run = q.SpawnRun(m, n0, n0 + 30, 2, 21)
    run.sample(init)
    run.propagate(200, dt, 10)
    assert run.status()["flags"] & q.FLAG_SPAWN_OVERFLOW
    assert n0 <= run.n_live() <= n0 + 30
    run2 = q.SpawnRun(m, n0, 100 * n0, 2, 2)
    run2.sample(init)
    run2.propagate(10, dt, 10)
    assert run2.status()["flags"] & q.FLAG_SPAWN_OVERFLOW == 0


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_fp32_spawn_nstate_observables_match_oracle(q, rep):
    """FP32 bulk spawning (one step per launch, the FP32 N_s-state walker
    arithmetic) against the oracle's FP64 spawning on the same walkers: the
    family means within the combined standard error, and walker lists of
    nearly the same length (FP32 decides differently only on rare
    near-threshold words)."""
    model, init, dt = _case(rep)
    n0, steps, stride = 3000, 120, 10
    cap = 60 * n0
    m = q.Model(model)
    run = q.SpawnRun(m, n0, cap, 13, steps // stride + 1, precision=q.PREC_FP32_BULK)
    run.sample(init)
    run.propagate(steps, dt, stride)
    obs = run.observables()
    assert run.status()["flags"] & (q.FLAG_NONFINITE | q.FLAG_SPAWN_OVERFLOW) == 0
    om = oracle.OracleModel(model)
    ref, n_live = oracle.run_spawn(om, oracle.OracleInit(om, init), 13, 0, n0, cap, dt, steps,
                                   stride)
    mean, se = oracle.finalize(ref, n0)
    nq = 4 * model["n_states"] ** 2
    diff = np.abs(obs[:, :nq] - mean)
    se2 = np.hypot(se, obs[:, nq:2 * nq])
    assert np.all(diff <= 3 * se2 + 1e-6), (diff / (se2 + 1e-300)).max()
    assert abs(run.n_live() - n_live[-1]) <= max(10, 0.01 * n_live[-1]), (run.n_live(), n_live[-1])
    assert run.n_live() > 1.2 * n0
    st = run.state()
    assert np.array_equal(np.unique(st["family"]), np.arange(n0))


def test_fp32_spawn_nstate_chunking_is_bitwise_invisible(q):
    model, init, dt = _case("adiabatic")
    n0, cap = 2000, 100_000
    outs = []
    for split in ((100,), (30, 70), (3, 97)):
        m = q.Model(model)
        run = q.SpawnRun(m, n0, cap, 4, 100 // 10 + 1, precision=q.PREC_FP32_BULK)
        run.sample(init)
        for k in split:
            run.propagate(k, dt, 10)
        outs.append((run.sums(), run.state()))
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0])
        for key in st:
            assert np.array_equal(st[key], outs[0][1][key]), key


def test_fp32_spawn_nstate_overflow_sets_flag(q):
    model, init, dt = _case("diabatic")
    n0 = 300
    m = q.Model(model)
    run = q.SpawnRun(m, n0, n0 + 30, 2, 21, precision=q.PREC_FP32_BULK)
    run.sample(init)
    run.propagate(200, dt, 10)
    assert run.status()["flags"] & q.FLAG_SPAWN_OVERFLOW
    assert n0 <= run.n_live() <= n0 + 30
