"""The larger N_s instantiations (five and eight states) of the diabatic
representation and of FP64 spawning: FP64 per trajectory against the oracle,
FP32 bulk against the FP64 path, spawning per walker against the oracle."""
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


def _model(ns, rep, seed=3, n=3):
    """Levels 0.4 apart with weak couplings (a spawning population grows
    2-4 fold in 100 steps of 0.01)."""
    rng = np.random.default_rng(seed)
    omega = rng.uniform(0.6, 1.5, size=n)
    E = np.diag(0.4 * np.arange(ns)) + 0.04 * (np.ones((ns, ns)) - np.eye(ns))
    K = np.zeros((n, ns, ns))
    for j in range(n):
        a = rng.normal(size=(ns, ns)) * 0.1
        K[j] = 0.5 * (a + a.T)
    m = wl._model(E, K, np.ones(n), omega, name=f"lvc{ns}-{rep}")
    m["repr"] = rep
    return m


def _state_to_oracle(om, st):
    s = oracle.State(om, len(st["m"]))
    for key in ("R", "P", "m", "phi", "alpha", "beta", "q"):
        getattr(s, key)[:] = st[key]
    if "U" in st:
        s.U[:] = st["U"]
    return s


@pytest.mark.parametrize("ns", [5, 8])
def test_diabatic_fp64_per_trajectory_parity_large_ns(q, ns):
    model = _model(ns, "diabatic")
    init = wl.sb_init(model, beta=3.0)
    m = q.Model(model)
    run = q.Run(m, 600, 7, q.PREC_FP64, 9)
    run.sample(init)
    om = oracle.OracleModel(model)
    flips, worst = 0, 0.0
    for s0 in range(0, 80, 40):
        ref = _state_to_oracle(om, run.state())
        oracle.advance(om, ref, 7, 0, s0, 40, 0.01)
        run.propagate(40, 0.01, 10)
        g = run.state()
        same = (g["alpha"] == ref.alpha) & (g["beta"] == ref.beta) & (g["q"] == ref.q)
        flips += int((~same).sum())
        for key, r in (("R", ref.R), ("P", ref.P), ("phi", ref.phi)):
            worst = max(worst, float((np.abs(g[key][same] - r[same])
                                      / np.maximum(np.abs(r[same]), 1.0)).max()))
        worst = max(worst, float((np.abs(g["m"][same] - ref.m[same]) / np.abs(ref.m[same])).max()))
    assert flips == 0 and worst < 1e-12, (flips, worst)
    g = run.state()
    assert np.any((g["alpha"] != 0) | (g["beta"] != 0))


@pytest.mark.parametrize("ns,rep", [(5, "diabatic"), (8, "diabatic"), (5, "adiabatic"),
                                    (8, "adiabatic")])
def test_fp32_matches_fp64_large_ns(q, ns, rep):
    model = _model(ns, rep)
    init = wl.sb_init(model, beta=3.0)
    m = q.Model(model)
    steps, stride, n = 200, 10, 100_000
    out = []
    for prec in (q.PREC_FP64, q.PREC_FP32_BULK):
        run = q.Run(m, n, 9, prec, steps // stride + 1)
        run.sample(init)
        run.propagate(steps, 0.01, stride)
        out.append(run.observables())
        assert run.status()["flags"] & q.FLAG_NONFINITE == 0
    a, b = out
    nq = 4 * ns * ns
    se = np.sqrt(a[:, nq:2 * nq] ** 2 + b[:, nq:2 * nq] ** 2)
    diff = np.abs(a[:, :nq] - b[:, :nq])
    assert np.all(diff <= 3.5 * se + 1e-9), (diff / (se + 1e-300)).max()
    ok = se.max(axis=1) < 1e-2
    assert ok.sum() >= 5 and diff[ok].max() < 1e-3


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_spawn_five_states_per_walker_parity(q, rep):
    model = _model(5, rep)
    init = wl.sb_init(model, beta=3.0)
    n0, cap, dt = 300, 300 * 60, 0.01
    m = q.Model(model)
    run = q.SpawnRun(m, n0, cap, 5, 11)
    run.sample(init)
    om = oracle.OracleModel(model)
    worst = 0.0
    for s0 in range(0, 100, 50):
        ck = run.state()
        ref = oracle.SpawnState(om, n0, cap)
        k = len(ck["m"])
        ref.n_live = k
        for key in ("R", "P", "m", "phi", "alpha", "beta", "q", "id", "family"):
            getattr(ref, key)[:k] = ck[key]
        if "U" in ck:
            ref.U[:k] = ck["U"]
        assert oracle.spawn_advance(om, ref, 5, s0, 50, dt) == 0
        run.propagate(50, dt, 10)
        g, r = run.state(), ref.live()
        assert len(g["m"]) == len(r["m"])
        for key in ("alpha", "beta", "q", "id", "family"):
            assert np.array_equal(g[key], r[key]), key
        for key in ("R", "P", "phi"):
            worst = max(worst, float((np.abs(g[key] - r[key]) / np.maximum(np.abs(r[key]), 1.0)).max()))
        worst = max(worst, float((np.abs(g["m"] - r["m"]) / np.abs(r["m"])).max()))
    assert worst < 1e-12, worst
    assert run.n_live() > 1.2 * n0
