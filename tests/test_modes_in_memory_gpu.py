"""FP32-bulk N_s-state models with more modes than a thread's registers hold
(more than 32 modes for N_s <= 4, more than 8 beyond), and below that limit
where it measured faster: the kernels' form that keeps R and P in the ensemble
buffer.  The same bits as the register form where both run (either forced by
QCL_OPT_MODES_IN_MEMORY), FP32 against the FP64 path and
against the oracle on the same walkers beyond the register limit, the sampler
for models whose K does not fit its parameter copy, spawning, and serving."""
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
    yield qcl
    qcl.set_option(qcl.OPT_MODES_IN_MEMORY, 0)


def _lvc(ns, n, rep, seed=5):
    """Levels 0.4 apart, off-diagonal couplings 0.04 in E, random symmetric
    K_j whose total strength does not grow with the mode count."""
    rng = np.random.default_rng(seed)
    omega = rng.uniform(0.6, 1.5, size=n)
    E = np.diag(0.4 * np.arange(ns)) + 0.04 * (np.ones((ns, ns)) - np.eye(ns))
    K = np.zeros((n, ns, ns))
    for j in range(n):
        a = rng.normal(size=(ns, ns)) * 0.12 * np.sqrt(6.0 / n)
        K[j] = 0.5 * (a + a.T)
    m = wl._model(E, K, np.ones(n), omega, name=f"lvc{ns}x{n}-{rep}")
    m["repr"] = rep
    return m


def _solve(q, model, n_traj, prec, seed, steps, stride, splits, mem=0, dt=0.01):
    q.set_option(q.OPT_MODES_IN_MEMORY, mem)
    try:
        run = q.Run(q.Model(model), n_traj, seed, prec, steps // stride + 1)
        run.sample(wl.sb_init(model, beta=3.0))
        for k in splits:
            run.propagate(k, dt, stride)
        return run
    finally:
        q.set_option(q.OPT_MODES_IN_MEMORY, 0)


@pytest.mark.parametrize("ns,n,rep", [(3, 6, "adiabatic"), (4, 32, "adiabatic"),
                                      (6, 8, "adiabatic"), (3, 6, "diabatic"),
                                      (5, 8, "diabatic"), (4, 32, "diabatic")])
def test_modes_in_memory_bitwise_equals_registers(q, ns, n, rep):
    """At a mode count the register form holds exactly (no padding modes), the
    modes-in-memory form gives the same walkers and sums bit for bit, over a
    chunk boundary and a ragged last tile."""
    model = _lvc(ns, n, rep)
    out = []
    for mem in (2, 1):  # registers, memory
        run = _solve(q, model, 5000 + 77, q.PREC_FP32_BULK, 3, 120, 10, (45, 75), mem=mem)
        assert run.status()["flags"] & q.FLAG_NONFINITE == 0
        out.append((run.sums(), run.state()))
    (s0, st0), (s1, st1) = out
    assert np.array_equal(s0, s1)
    for key in st0:
        assert np.array_equal(st0[key], st1[key]), key
    moved = (st0["alpha"] != 0) | (st0["beta"] != 0)
    assert moved.any()


_MANY = [(3, 40, "adiabatic"), (3, 40, "diabatic"), (6, 12, "adiabatic"),
         (8, 10, "diabatic"), (5, 64, "adiabatic"), (8, 40, "adiabatic"),
         (4, 256, "diabatic")]


@pytest.mark.parametrize("ns,n,rep", _MANY)
def test_many_modes_fp32_matches_fp64_and_oracle(q, ns, n, rep):
    """Beyond the register limit: FP32-bulk means within the combined standard
    error of the FP64 path (and within 1e-3 where both resolve them), and the
    same walkers (seed, ids, Philox streams) through the oracle within its
    standard error."""
    model = _lvc(ns, n, rep)
    steps, stride, nw = 200, 10, 100_000
    a = _solve(q, model, nw, q.PREC_FP64, 9, steps, stride, (steps,)).observables()
    rb = _solve(q, model, nw, q.PREC_FP32_BULK, 9, steps, stride, (steps,))
    b = rb.observables()
    assert rb.status()["flags"] & q.FLAG_NONFINITE == 0
    nq = 4 * ns * ns
    se = np.sqrt(a[:, nq:2 * nq] ** 2 + b[:, nq:2 * nq] ** 2)
    diff = np.abs(a[:, :nq] - b[:, :nq])
    assert np.all(diff <= 3.5 * se + 1e-9), (diff / (se + 1e-300)).max()
    ok = se.max(axis=1) < 1e-2
    assert ok.sum() >= 3 and diff[ok].max() < 1e-3
    nm = 3000
    c = _solve(q, model, nm, q.PREC_FP32_BULK, 4, steps, stride, (steps,)).observables()
    om = oracle.OracleModel(model)
    ref, _ = oracle.run(om, oracle.OracleInit(om, wl.sb_init(model, beta=3.0)), 4, 0, nm, 0.01,
                        steps, stride)
    mean, se_o = oracle.finalize(ref, nm)
    d = np.abs(c[:, :nq] - mean)
    assert np.all(d <= 3.5 * se_o + 1e-9), (d / (se_o + 1e-300)).max()
    ok = se_o.max(axis=1) < 1e-2
    if ok.any():
        assert d[ok].max() < 1e-3


@pytest.mark.parametrize("ns,n,rep", [(3, 60, "adiabatic"), (8, 10, "diabatic")])
def test_fp32_sampler_reads_large_k_from_the_model(q, ns, n, rep):
    """n N_s^2 above the sampler's parameter copy of K (512 values): the FP32
    sample against the oracle's FP64 sample of the same walkers."""
    assert n * ns * ns > 512
    model = _lvc(ns, n, rep)
    nw = 4000
    st = _solve(q, model, nw, q.PREC_FP32_BULK, 21, 10, 10, ()).state()
    om = oracle.OracleModel(model)
    ref = oracle.sample(om, oracle.OracleInit(om, wl.sb_init(model, beta=3.0)), 21, 0, nw)
    for key, r in (("R", ref.R), ("P", ref.P)):
        err = np.abs(st[key] - r) / np.maximum(np.abs(r), 1.0)
        assert err.max() < 1e-5, (key, err.max())
    same = (st["alpha"] == ref.alpha) & (st["beta"] == ref.beta)
    assert same.mean() > 0.995, same.mean()
    # (the weight is a ratio of FP32 decomposition products: 1e-4 relative)
    assert np.allclose(st["m"][same], ref.m[same], rtol=1e-4)


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_spawn_modes_in_memory_bitwise_equals_registers(q, rep):
    model = _lvc(3, 4, rep, seed=13)
    n0, cap = 1500, 60_000
    out = []
    for mem in (2, 1):  # registers, memory
        q.set_option(q.OPT_MODES_IN_MEMORY, mem)
        try:
            run = q.SpawnRun(q.Model(model), n0, cap, 5, 11, precision=q.PREC_FP32_BULK)
            run.sample(wl.sb_init(model, beta=3.0))
            run.propagate(40, 0.01, 10)
            run.propagate(60, 0.01, 10)
        finally:
            q.set_option(q.OPT_MODES_IN_MEMORY, 0)
        out.append((run.sums(), run.state(), run.n_live()))
    assert out[0][2] == out[1][2] and out[0][2] > n0
    assert np.array_equal(out[0][0], out[1][0])
    for key in out[0][1]:
        assert np.array_equal(out[0][1][key], out[1][1][key]), key


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_spawn_many_modes_fp32_matches_oracle(q, rep):
    """FP32 spawning of a 12-mode three-state model (past the 8 modes held in
    registers) against the oracle's FP64 spawning of the same walkers."""
    model = _lvc(3, 12, rep, seed=13)
    init = wl.sb_init(model, beta=3.0)
    n0, steps, stride = 3000, 120, 10
    cap = 60 * n0
    run = q.SpawnRun(q.Model(model), n0, cap, 13, steps // stride + 1,
                     precision=q.PREC_FP32_BULK)
    run.sample(init)
    run.propagate(steps, 0.01, stride)
    assert run.status()["flags"] & (q.FLAG_NONFINITE | q.FLAG_SPAWN_OVERFLOW) == 0
    obs = run.observables()
    om = oracle.OracleModel(model)
    ref, n_live = oracle.run_spawn(om, oracle.OracleInit(om, init), 13, 0, n0, cap, 0.01, steps,
                                   stride)
    mean, se = oracle.finalize(ref, n0)
    nq = 4 * 9
    diff = np.abs(obs[:, :nq] - mean)
    se2 = np.hypot(se, obs[:, nq:2 * nq])
    assert np.all(diff <= 3.5 * se2 + 1e-6), (diff / (se2 + 1e-300)).max()
    assert abs(run.n_live() - n_live[-1]) <= max(10, 0.01 * n_live[-1])
    assert run.n_live() > 1.2 * n0


def test_served_many_modes_equals_single_solve(q):
    model = _lvc(3, 40, "adiabatic")
    n, steps, stride = 30_000, 150, 10
    single = _solve(q, model, n, q.PREC_FP32_BULK, 21, steps, stride, (steps,)).observables()
    srv = q.Server(1 << 30, quantum_steps=60)
    rid = srv.submit(dict(model=model, init=wl.sb_init(model, beta=3.0), n_traj=n, seed=21,
                          n_steps=steps, dt=0.01, out_stride=stride))
    st, obs = srv.wait(rid)
    srv.close()
    assert st == q.REQ_DONE
    assert np.array_equal(obs, single)
