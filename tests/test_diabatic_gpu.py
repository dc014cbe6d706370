"""Diabatic representation on the GPU (through the C ABI) against the FP64
oracle: FP64 per-trajectory parity at 1e-12 with identical transitions and
quarter turns, FP32-bulk ensemble observables within 3 standard errors, the
pure-dephasing closed form at eps = 0 (the crossing regime), bitwise chunk
invariance, and the served path."""
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


def _dia(cfg):
    c = copy.deepcopy(cfg)
    c["model"]["repr"] = "diabatic"
    return c


def _oracle_state(om, st):
    s = oracle.State(om, len(st["m"]))
    s.R[:] = st["R"]
    s.P[:] = st["P"]
    s.m[:] = st["m"]
    s.phi[:] = st["phi"]
    s.alpha[:] = st["alpha"]
    s.beta[:] = st["beta"]
    s.q[:] = st["q"]
    return s


def _run(q, cfg, n_traj, prec, n_steps, stride, seed=0, offset=0):
    m = q.Model(cfg["model"])
    run = q.Run(m, n_traj, seed, prec, n_steps // stride + 1, traj_id_offset=offset)
    run.sample(cfg["init"])
    return m, run


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_dia_sample_matches_oracle(q, prec_name):
    cfg = _dia(wl.config(2))
    cfg["init"]["rho_el0"] = np.array([[0.6, 0.3], [0.3, 0.4]])
    prec = q.PREC_FP64 if prec_name == "fp64" else q.PREC_FP32_BULK
    n = 3000
    m, run = _run(q, cfg, n, prec, 10, 10, seed=9, offset=77)
    st = run.state()
    om = oracle.OracleModel(cfg["model"])
    ref = oracle.sample(om, oracle.OracleInit(om, cfg["init"]), 9, 77, n)
    assert np.array_equal(st["alpha"], ref.alpha) and np.array_equal(st["beta"], ref.beta)
    assert np.all(st["q"] == 0)
    w = st["m"] * 2.0 ** st["m_exp"]
    tol = 1e-13 if prec == q.PREC_FP64 else 1e-6
    assert np.allclose(w, ref.m, rtol=tol)
    # all four pairs are drawn (the coherences of rho_el0 are sampled directly)
    assert len(set(zip(st["alpha"], st["beta"]))) == 4


def _segment_parity(q, cfg, n_traj, n_steps, seg, seed):
    m, run = _run(q, cfg, n_traj, q.PREC_FP64, n_steps, cfg["out_stride"], seed=seed)
    om = oracle.OracleModel(cfg["model"])
    worst, flips, hops = {}, 0, 0
    for s0 in range(0, n_steps, seg):
        ck = run.state()
        ref = _oracle_state(om, ck)
        oracle.advance(om, ref, seed, 0, s0, seg, cfg["dt"])
        run.propagate(seg, cfg["dt"], cfg["out_stride"])
        g = run.state()
        same = (g["alpha"] == ref.alpha) & (g["beta"] == ref.beta) & (g["q"] == ref.q)
        flips += int((~same).sum())
        hops += int(((g["q"] != ck["q"]) & same).sum())
        for key, r in (("R", ref.R), ("P", ref.P), ("phi", ref.phi), ("m", ref.m)):
            x, y = g[key][same], r[same]
            den = np.abs(y) + 1e-300 if key == "m" else np.maximum(np.abs(y), 1.0)
            err = np.abs(x - y) / den
            worst[key] = max(worst.get(key, 0.0), float(err.max()) if err.size else 0.0)
    st = run.status()
    assert st["step"] == n_steps and st["flags"] == 0
    return worst, flips, hops


@pytest.mark.parametrize("cfg_id,n,steps,seg", [(1, 4000, 600, 100), (2, 3000, 400, 50),
                                                (3, 3000, 400, 50)])
def test_fp64_dia_per_trajectory_parity(q, cfg_id, n, steps, seg):
    cfg = _dia(wl.config(cfg_id))
    worst, flips, hops = _segment_parity(q, cfg, n, steps, seg, 5)
    assert flips <= 1
    assert hops > 100  # transitions (with their quarter turns) were exercised
    assert max(worst.values()) < 1e-12, worst


def test_fp64_dia_observables_match_oracle(q):
    cfg = _dia(wl.config(2))
    n, steps, stride = 2000, 400, 10
    m, run = _run(q, cfg, n, q.PREC_FP64, steps, stride, seed=4)
    run.propagate(steps, cfg["dt"], stride)
    sums = run.sums()
    om = oracle.OracleModel(cfg["model"])
    ref, _ = oracle.run(om, oracle.OracleInit(om, cfg["init"]), 4, 0, n, cfg["dt"], steps, stride)
    scale = np.sqrt(n * np.abs(ref[:, 16:])) + 1e-300
    err = np.abs(sums[:, :16] - ref[:, :16]) / scale
    assert err.max() < 1e-10, err.max()


def test_fp32_dia_pure_dephasing_at_eps0(q):
    """Delta = 0, eps = 0: the diabatic levels cross at every bath fluctuation;
    the coherence is the Gaussian characteristic function of the phase."""
    model = pins._dephasing_model(eps=0.0)
    model["repr"] = "diabatic"
    init = pins._plus_init(model, beta=2.0)
    cfg = {"model": model, "init": init, "dt": 0.01, "out_stride": 40}
    n, steps = 200_000, 400
    m, run = _run(q, cfg, n, q.PREC_FP32_BULK, steps, 40, seed=5)
    run.propagate(steps, 0.01, 40)
    obs = run.observables()
    disc, _ = pins._dephasing_closed_form(model, init, 0.01, np.arange(0, steps + 1, 40), 0.0)
    r01 = obs[:, 2] + 1j * obs[:, 3]
    s01 = obs[:, 16 + 2] + 1j * obs[:, 16 + 3]
    assert np.all(np.abs(r01.real - 0.5 * disc.real) < 4 * s01.real + 2e-6)
    assert np.all(np.abs(r01.imag - 0.5 * disc.imag) < 4 * s01.imag + 2e-6)
    assert abs(disc[-1]) < 0.9
    st = run.state()
    assert np.all(st["q"] == 0)  # no transition fired


def test_fp32_dia_chunking_and_launch_shape_bitwise(q):
    cfg = _dia(wl.config(3))
    n, steps, stride = 50_000, 400, 20
    outs = []
    for split, cap in (((400,), 0), ((130, 135, 135), 0), ((400,), 7), ((1, 399), 300)):
        q.set_option(q.OPT_GRID_CAP, cap)
        m, run = _run(q, cfg, n, q.PREC_FP32_BULK, steps, stride, seed=4)
        for k in split:
            run.propagate(k, cfg["dt"], stride)
        outs.append((run.sums(), run.state()))
    q.set_option(q.OPT_GRID_CAP, 0)
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0])
        for k in st:
            assert np.array_equal(st[k], outs[0][1][k]), k
    assert np.any(outs[0][1]["q"] != 0)


def test_served_dia_request_matches_single_solve(q):
    cfg = _dia(wl.config(2))
    n, steps = 60_000, 400
    srv = q.Server(1 << 30, quantum_steps=150)
    rid = srv.submit(dict(model=cfg["model"], init=cfg["init"], n_traj=n, seed=7, n_steps=steps,
                          dt=cfg["dt"], out_stride=cfg["out_stride"]))
    st, served = srv.wait(rid)
    srv.close()
    assert st == q.REQ_DONE
    m, run = _run(q, cfg, n, q.PREC_FP32_BULK, steps, cfg["out_stride"], seed=7)
    run.propagate(steps, cfg["dt"], cfg["out_stride"])
    single = run.observables()
    assert np.array_equal(served[:, :32], single[:, :32])
