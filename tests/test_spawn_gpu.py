"""Trajectory spawning on the GPU (FP64, through the C ABI) against the oracle:
per-walker parity (same walker list, ids and families; R, P, phi, m to
1e-12), family-summed observables, bitwise identity with the no-spawn path
when nothing can fire, chunk invariance, and the capacity-overflow flag."""
import copy

import numpy as np
import pytest

import oracle
from paper_2608_14544_gb300 import workloads as wl
from tests import test_oracle_pins as pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch

    from paper_2608_14544_gb300 import build, qcl

    build.build()
    oracle.build()
    torch.cuda.set_device(0)
    return qcl


def _cfg(cfg_id, rep):
    c = copy.deepcopy(wl.config(cfg_id))
    c["model"]["repr"] = rep
    return c


def _oracle_from_gpu(om, st, n0, cap):
    s = oracle.SpawnState(om, n0, cap)
    k = len(st["m"])
    s.n_live = k
    for key in ("R", "P", "m", "phi", "alpha", "beta", "q", "id", "family"):
        getattr(s, key)[:k] = st[key]
    return s


@pytest.mark.parametrize("cfg_id,rep,n0,steps,seg", [(1, "adiabatic", 1500, 400, 50),
                                                     (2, "diabatic", 800, 200, 40),
                                                     (3, "adiabatic", 600, 200, 40)])
def test_spawn_per_walker_parity(q, cfg_id, rep, n0, steps, seg):
    cfg = _cfg(cfg_id, rep)
    cap = 60 * n0
    m = q.Model(cfg["model"])
    run = q.SpawnRun(m, n0, cap, 5, steps // cfg["out_stride"] + 1, traj_id_offset=100)
    run.sample(cfg["init"])
    om = oracle.OracleModel(cfg["model"])
    ref0 = oracle.spawn_sample(om, oracle.OracleInit(om, cfg["init"]), 5, 100, n0, cap)
    st = run.state()
    for key in ("alpha", "beta", "q", "id", "family"):
        assert np.array_equal(st[key], ref0.live()[key]), key
    worst = {}
    for s0 in range(0, steps, seg):
        ck = run.state()
        ref = _oracle_from_gpu(om, ck, n0, cap)
        assert oracle.spawn_advance(om, ref, 5, s0, seg, cfg["dt"]) == 0
        run.propagate(seg, cfg["dt"], cfg["out_stride"])
        g = run.state()
        r = ref.live()
        assert len(g["m"]) == len(r["m"]), (s0, len(g["m"]), len(r["m"]))
        for key in ("alpha", "beta", "q", "id", "family"):
            assert np.array_equal(g[key], r[key]), (s0, key)
        for key in ("R", "P", "phi", "m"):
            den = np.abs(r[key]) + 1e-300 if key == "m" else np.maximum(np.abs(r[key]), 1.0)
            worst[key] = max(worst.get(key, 0.0), float((np.abs(g[key] - r[key]) / den).max()))
    assert max(worst.values()) < 1e-12, worst
    assert run.n_live() > 1.2 * n0  # children were spawned
    assert run.status()["flags"] & q.FLAG_SPAWN_OVERFLOW == 0


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_spawn_observables_match_oracle(q, rep):
    cfg = _cfg(1, rep)
    n0, steps, stride, cap = 2000, 300, 10, 400_000
    m = q.Model(cfg["model"])
    run = q.SpawnRun(m, n0, cap, 3, steps // stride + 1)
    run.sample(cfg["init"])
    run.propagate(steps, cfg["dt"], stride)
    sums = run.sums()
    om = oracle.OracleModel(cfg["model"])
    ref, n_live = oracle.run_spawn(om, oracle.OracleInit(om, cfg["init"]), 3, 0, n0, cap,
                                   cfg["dt"], steps, stride)
    scale = np.sqrt(n0 * np.abs(ref[:, 16:])) + 1e-300
    err = np.abs(sums[:, :16] - ref[:, :16]) / scale
    assert err.max() < 1e-10, err.max()
    assert np.allclose(sums[:, 16:], ref[:, 16:], rtol=1e-9, atol=1e-12)
    assert run.n_live() == n_live[-1]
    obs = run.observables()
    assert np.allclose(obs[:, 34], n0)  # means and errors are over the n0 families


def test_spawn_without_coupling_equals_no_spawn_bits(q):
    model = pins._dephasing_model()
    init = pins._plus_init(model, beta=2.0)
    cfg = {"model": model, "init": init}
    n0, steps, stride = 3000, 200, 20
    m = q.Model(model)
    sp = q.SpawnRun(m, n0, n0, 9, steps // stride + 1)
    sp.sample(init)
    sp.propagate(steps, 0.01, stride)
    run = q.Run(m, n0, 9, q.PREC_FP64, steps // stride + 1)
    run.sample(init)
    run.propagate(steps, 0.01, stride)
    assert sp.n_live() == n0
    assert np.array_equal(sp.sums(), run.sums())
    a, b = sp.state(), run.state()
    for key in ("R", "P", "phi", "m", "alpha", "beta"):
        assert np.array_equal(a[key], b[key]), key


def test_spawn_chunking_is_bitwise_invisible(q):
    cfg = _cfg(1, "adiabatic")
    n0, cap = 1000, 200_000
    outs = []
    for split in ((200,), (70, 130), (1, 99, 100)):
        m = q.Model(cfg["model"])
        run = q.SpawnRun(m, n0, cap, 4, 200 // 10 + 1)
        run.sample(cfg["init"])
        for k in split:
            run.propagate(k, cfg["dt"], 10)
        outs.append((run.sums(), run.state()))
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0])
        for key in st:
            assert np.array_equal(st[key], outs[0][1][key]), key


def test_spawn_overflow_sets_flag(q):
    cfg = _cfg(1, "adiabatic")
    n0 = 500
    m = q.Model(cfg["model"])
    run = q.SpawnRun(m, n0, n0 + 40, 2, 31)
    run.sample(cfg["init"])
    run.propagate(300, cfg["dt"], 10)
    st = run.status()
    assert st["flags"] & q.FLAG_SPAWN_OVERFLOW
    assert n0 <= run.n_live() <= n0 + 40
    # the context stays usable
    run2 = q.SpawnRun(m, n0, 100 * n0, 2, 2)
    run2.sample(cfg["init"])
    run2.propagate(10, cfg["dt"], 10)
    assert run2.status()["flags"] & q.FLAG_SPAWN_OVERFLOW == 0


# ------------------------------------------------------------ FP32 spawning --
@pytest.mark.parametrize("cfg_id,rep,n0,steps", [(1, "adiabatic", 6000, 300),
                                                 (2, "adiabatic", 4000, 200),
                                                 (2, "diabatic", 4000, 200),
                                                 (3, "adiabatic", 3000, 200)])
def test_fp32_spawn_observables_match_oracle(q, cfg_id, rep, n0, steps):
    cfg = _cfg(cfg_id, rep)
    stride, cap = cfg["out_stride"], 400 * n0
    m = q.Model(cfg["model"])
    run = q.SpawnRun(m, n0, cap, 13, steps // stride + 1, precision=q.PREC_FP32_BULK)
    run.sample(cfg["init"])
    run.propagate(steps, cfg["dt"], stride)
    obs = run.observables()
    assert run.status()["flags"] == 0
    om = oracle.OracleModel(cfg["model"])
    ref, n_live = oracle.run_spawn(om, oracle.OracleInit(om, cfg["init"]), 13, 0, n0, cap,
                                   cfg["dt"], steps, stride)
    mean, se = oracle.finalize(ref, n0)
    diff = np.abs(obs[:, :16] - mean)
    # both estimate the same expectation; their errors are independent only up
    # to the shared random streams, so the combined SE bounds the difference
    se2 = np.hypot(se, obs[:, 16:32])
    assert np.all(diff <= 3 * se2 + 1e-6), (diff / (se2 + 1e-300)).max()
    # the walker lists agree closely (decisions in FP32 against FP64 differ only
    # for rare near-threshold words)
    assert abs(run.n_live() - n_live[-1]) <= max(5, 0.002 * n_live[-1])
    assert run.n_live() > 1.1 * n0


def test_fp32_spawn_chunking_is_bitwise_invisible(q):
    cfg = _cfg(2, "adiabatic")
    n0, cap = 3000, 1_500_000
    outs = []
    for split in ((200,), (70, 130), (3, 197)):
        m = q.Model(cfg["model"])
        run = q.SpawnRun(m, n0, cap, 4, 200 // 10 + 1, precision=q.PREC_FP32_BULK)
        run.sample(cfg["init"])
        for k in split:
            run.propagate(k, cfg["dt"], 10)
        outs.append((run.sums(), run.state()))
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0])
        for key in st:
            assert np.array_equal(st[key], outs[0][1][key]), key


def test_fp32_spawn_overflow_sets_flag(q):
    cfg = _cfg(1, "adiabatic")
    n0 = 500
    m = q.Model(cfg["model"])
    run = q.SpawnRun(m, n0, n0 + 40, 2, 31, precision=q.PREC_FP32_BULK)
    run.sample(cfg["init"])
    run.propagate(300, cfg["dt"], 10)
    assert run.status()["flags"] & q.FLAG_SPAWN_OVERFLOW
    assert n0 <= run.n_live() <= n0 + 40


@pytest.mark.parametrize("cfg_id,rep", [(2, "adiabatic"), (2, "diabatic"), (3, "adiabatic")])
def test_fp32_spawn_modes_in_memory_bitwise_equals_registers(q, cfg_id, rep):
    """The spawning step's form that keeps R and P in memory (taken beyond 32
    modes, forced here by QCL_OPT_MODES_IN_MEMORY = 1) against the register
    form: the same walkers, families and sums, bit for bit."""
    cfg = _cfg(cfg_id, rep)
    n0, cap = 2000, 400_000
    outs = []
    for mem in (0, 1):
        q.set_option(q.OPT_MODES_IN_MEMORY, mem)
        try:
            run = q.SpawnRun(q.Model(cfg["model"]), n0, cap, 6, 16, precision=q.PREC_FP32_BULK)
            run.sample(cfg["init"])
            run.propagate(60, cfg["dt"], 10)
            run.propagate(90, cfg["dt"], 10)
        finally:
            q.set_option(q.OPT_MODES_IN_MEMORY, 0)
        outs.append((run.sums(), run.state(), run.n_live()))
    assert outs[0][2] == outs[1][2] and outs[0][2] > n0
    assert np.array_equal(outs[0][0], outs[1][0])
    for key in outs[0][1]:
        assert np.array_equal(outs[0][1][key], outs[1][1][key]), key


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_fp32_spawn_many_modes_match_oracle(q, rep):
    """FP32 spawning of a 40-mode two-state model (past the 32 modes held in
    registers) against the oracle's FP64 spawning of the same walkers."""
    model = wl.random_lvc2(40, seed=40, scale=0.1)
    model["repr"] = rep
    init = wl.sb_init(model, beta=2.0)
    n0, steps, stride, dt = 3000, 150, 10, 0.01
    cap = 200 * n0
    run = q.SpawnRun(q.Model(model), n0, cap, 13, steps // stride + 1,
                     precision=q.PREC_FP32_BULK)
    run.sample(init)
    run.propagate(steps, dt, stride)
    assert run.status()["flags"] == 0
    obs = run.observables()
    om = oracle.OracleModel(model)
    ref, n_live = oracle.run_spawn(om, oracle.OracleInit(om, init), 13, 0, n0, cap, dt, steps,
                                   stride)
    mean, se = oracle.finalize(ref, n0)
    diff = np.abs(obs[:, :16] - mean)
    se2 = np.hypot(se, obs[:, 16:32])
    # (256 comparisons: 3.5 combined standard errors)
    assert np.all(diff <= 3.5 * se2 + 1e-6), (diff / (se2 + 1e-300)).max()
    assert abs(run.n_live() - n_live[-1]) <= max(5, 0.002 * n_live[-1])
    assert run.n_live() > 1.1 * n0
