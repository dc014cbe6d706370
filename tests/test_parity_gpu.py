"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

FP64 path: per trajectory to 1e-12 relative over deterministic segments, each
comparison restarted from the GPU's own checkpoint, with identical transition
decisions.  FP32-bulk path: ensemble observables within 3 standard errors and
1e-3 absolute.  Bitwise invariance of results under chunking and launch shape.
"""
import math

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


def _gpu_run(q, cfg, n_traj, prec, n_steps, stride, seed=0, offset=0, init=None, model=None):
    m = q.Model(model or cfg["model"])
    run = q.Run(m, n_traj, seed, prec, n_steps // stride + 1, traj_id_offset=offset)
    run.sample(init or cfg["init"])
    return m, run


# ------------------------------------------------------------------ sampling --
@pytest.mark.parametrize("n_traj", [1, 255, 256, 257, 1000])
def test_fp64_sample_matches_oracle(q, n_traj):
    cfg = wl.config(2)
    m, run = _gpu_run(q, cfg, n_traj, q.PREC_FP64, 10, 10, seed=7, offset=12345)
    st = run.state()
    om = oracle.OracleModel(cfg["model"])
    ref = oracle.sample(om, oracle.OracleInit(om, cfg["init"]), 7, 12345, n_traj)
    assert np.allclose(st["R"], ref.R, rtol=1e-13, atol=1e-14)
    assert np.allclose(st["P"], ref.P, rtol=1e-13, atol=1e-14)
    assert np.array_equal(st["alpha"], ref.alpha) and np.array_equal(st["beta"], ref.beta)
    assert np.allclose(st["m"], ref.m, rtol=1e-13)
    assert np.all(st["phi"] == 0.0)


def test_fp32_sample_matches_oracle(q):
    cfg = wl.config(2)
    n = 4096
    m, run = _gpu_run(q, cfg, n, q.PREC_FP32_BULK, 10, 10, seed=3)
    st = run.state()
    om = oracle.OracleModel(cfg["model"])
    ref = oracle.sample(om, oracle.OracleInit(om, cfg["init"]), 3, 0, n)
    scale = np.abs(ref.R).max()
    assert np.abs(st["R"] - ref.R).max() < 1e-5 * scale
    assert np.abs(st["P"] - ref.P).max() < 1e-5 * np.abs(ref.P).max()
    same = (st["alpha"] == ref.alpha) & (st["beta"] == ref.beta)
    assert same.mean() > 0.999
    # m0 = rho_ad / p_hat: a one-unit change of a 24-bit threshold between the
    # FP32 and FP64 evaluations moves m0 by 1/T, large only for rare small-T pairs
    rel = np.abs(st["m"][same] * 2.0 ** st["m_exp"][same] - ref.m[same]) / np.abs(ref.m[same])
    assert np.median(rel) < 1e-6 and np.mean(rel > 1e-5) < 1e-3


# ------------------------------------------------- FP64 per-trajectory parity --
def _segment_parity(q, cfg, n_traj, n_steps, seg, seed):
    m, run = _gpu_run(q, cfg, n_traj, q.PREC_FP64, n_steps, cfg["out_stride"], seed=seed)
    om = oracle.OracleModel(cfg["model"])
    worst = {}
    flips = 0
    for s0 in range(0, n_steps, seg):
        ck = run.state()
        ref = _oracle_state(om, ck)
        oracle.advance(om, ref, seed, 0, s0, seg, cfg["dt"])
        run.propagate(seg, cfg["dt"], cfg["out_stride"])
        g = run.state()
        same = (g["alpha"] == ref.alpha) & (g["beta"] == ref.beta) & (g["q"] == ref.q)
        flips += int((~same).sum())
        for key, r in (("R", ref.R), ("P", ref.P), ("phi", ref.phi), ("m", ref.m)):
            x = g[key][same]
            y = r[same]
            den = np.maximum(np.abs(y), 1.0 if key != "m" else 1e-300)
            err = np.abs(x - y) / (den if key != "m" else np.abs(y) + 1e-300)
            worst[key] = max(worst.get(key, 0.0), float(err.max()) if err.size else 0.0)
    st = run.status()
    assert st["step"] == n_steps and (st["flags"] & q.FLAG_STEP_MISMATCH) == 0
    return worst, flips


def test_fp64_per_trajectory_parity_config1(q):
    cfg = wl.config(1)
    worst, flips = _segment_parity(q, cfg, cfg["n_traj"], cfg["n_steps"], 100, cfg["seed"])
    assert flips == 0
    assert max(worst.values()) < 1e-12, worst


def test_fp64_per_trajectory_parity_vibronic(q):
    cfg = wl.config(3)
    worst, flips = _segment_parity(q, cfg, 3000, 400, 50, 5)
    assert flips <= 1
    assert max(worst.values()) < 1e-12, worst


def test_fp64_per_trajectory_parity_config2(q):
    """The benchmark model (3-mode ohmic spin-boson, thermal), adiabatic."""
    cfg = wl.config(2)
    worst, flips = _segment_parity(q, cfg, 4000, cfg["n_steps"], 100, cfg["seed"])
    assert flips == 0
    assert max(worst.values()) < 1e-12, worst


def _capped(rep):
    """The 1-mode model with a small p_max: the two events' probabilities (dt
    |d.P/M| each, up to about 0.007, or dt |V_01| / hbar = 0.005) sum above the
    cap (0.001 adiabatic, 0.004 diabatic) and are scaled down together at most
    walker-steps (checked)."""
    cfg = wl.config(1)
    cfg["model"]["p_max"] = 0.001 if rep == "adiabatic" else 0.004
    cfg["model"]["repr"] = rep
    return cfg


def _capped_fraction(cfg, st, n=500):
    om = oracle.OracleModel(cfg["model"])
    tmax = math.floor(cfg["model"]["p_max"] * 2**24)
    hit = 0
    for i in range(n):
        a, b = int(st["alpha"][i]), int(st["beta"][i])
        if cfg["model"]["repr"] == "diabatic":
            T = oracle.events_dia(om, st["R"][i], a, b, cfg["dt"])[4]
        else:
            e, U, _ = oracle.adiabatic(om, st["R"][i])
            T = oracle.events(om, st["P"][i], e, U, a, b, cfg["dt"])[3]
        hit += int(T.astype(np.int64).sum()) >= tmax - len(T)
    return hit / n


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_capped_probabilities_fp64_parity_and_fp32_matched_ensemble(q, rep):
    """The capped branch of the transition rule on the GPU: FP64 per trajectory
    (identical decisions, 1e-12) and the FP32-bulk ensemble of the same walkers
    within 1e-3 and 3 SE of the oracle."""
    cfg = _capped(rep)
    worst, flips = _segment_parity(q, cfg, 3000, 600, 100, 5)
    assert flips == 0
    assert max(worst.values()) < 1e-12, worst
    n, steps, stride = 1 << 15, cfg["n_steps"], cfg["out_stride"]
    m, run = _gpu_run(q, cfg, n, q.PREC_FP32_BULK, steps, stride, seed=5)
    assert _capped_fraction(cfg, run.state()) > 0.5
    run.propagate(steps, cfg["dt"], stride)
    obs = run.observables()
    om = oracle.OracleModel(cfg["model"])
    ref, _ = oracle.run(om, oracle.OracleInit(om, cfg["init"]), 5, 0, n, cfg["dt"], steps, stride)
    mean, se = oracle.finalize(ref, n)
    diff = np.abs(obs[:, :16] - mean)
    assert np.all(diff <= 3 * se + 1e-7)
    res = se < 1e-2
    assert res.any(axis=1).sum() >= 5 and diff[res].max() < 1e-3
    assert _capped_fraction(cfg, run.state()) > 0.5


def test_fp64_observables_match_oracle(q):
    cfg = wl.config(1)
    n, steps = 2000, 1000
    m, run = _gpu_run(q, cfg, n, q.PREC_FP64, steps, 10)
    run.propagate(steps, cfg["dt"], 10)
    sums = run.sums()
    om = oracle.OracleModel(cfg["model"])
    ref, _ = oracle.run(om, oracle.OracleInit(om, cfg["init"]), 0, 0, n, cfg["dt"], steps, 10)
    scale = np.sqrt(n * np.abs(ref[:, 16:])) + 1e-300
    err = np.abs(sums[:, :16] - ref[:, :16]) / scale
    assert err.max() < 1e-10, err.max()
    obs = run.observables()
    mean, se = oracle.finalize(ref, n)
    assert np.allclose(obs[:, :16], mean, rtol=1e-9, atol=1e-12)
    assert np.allclose(obs[:, 16:32], se, rtol=1e-6, atol=1e-12)
    assert np.allclose(obs[:, 34], n)


# -------------------------------------------- FP32-bulk ensemble-level parity --
def test_fp32_bulk_vs_fp64_large_ensemble(q):
    cfg = wl.config(2)
    n, steps, stride = 1 << 20, 2000, 10
    res = {}
    for prec in (q.PREC_FP64, q.PREC_FP32_BULK):
        m, run = _gpu_run(q, cfg, n, prec, steps, stride, seed=2)
        run.propagate(steps, cfg["dt"], stride)
        res[prec] = run.observables()
    a, b = res[q.PREC_FP64], res[q.PREC_FP32_BULK]
    se = np.sqrt(a[:, 16:32] ** 2 + b[:, 16:32] ** 2)
    diff = np.abs(a[:, :16] - b[:, :16])
    assert np.all(np.isfinite(b[:, :32]))
    assert np.all(diff <= 3 * se + 1e-9), (diff / (se + 1e-300)).max()
    # the absolute bound applies where the estimator itself resolves 1e-3: the
    # weights of the no-spawn estimator grow like exp(2 int |P d/M| dt)
    # (the walkers are matched: same Philox streams, so early on the two paths
    # differ by far less than one standard error)
    resolved = se.max(axis=1) < 1e-2
    assert resolved.sum() >= 10
    assert diff[resolved].max() < 1e-3


# ----------------------------------------------------------- invariances --
def test_fp32_chunking_and_launch_shape_are_bitwise_invisible(q):
    cfg = wl.config(2)
    n, steps, stride = 50_000, 400, 10
    outs = []
    for split, cap in (((400,), 0), ((130, 135, 135), 0), ((400,), 7), ((1, 399), 300)):
        q.set_option(q.OPT_GRID_CAP, cap)
        m, run = _gpu_run(q, cfg, n, q.PREC_FP32_BULK, steps, stride, seed=4)
        for k in split:
            run.propagate(k, cfg["dt"], stride)
        outs.append((run.sums(), run.state()))
    q.set_option(q.OPT_GRID_CAP, 0)
    for sums, st in outs[1:]:
        assert np.array_equal(sums, outs[0][0])
        for k in st:
            assert np.array_equal(st[k], outs[0][1][k]), k


def test_fp64_chunking_is_bitwise_invisible(q):
    cfg = wl.config(1)
    outs = []
    for split in ((200,), (70, 130)):
        m, run = _gpu_run(q, cfg, 3000, q.PREC_FP64, 200, 10, seed=9)
        for k in split:
            run.propagate(k, cfg["dt"], 10)
        outs.append(run.sums())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", [0, 1])
def test_zero_coupling_populations_constant(q, prec):
    model = pins._dephasing_model()
    init = wl.sb_init(model, beta=2.0)
    m, run = _gpu_run(q, None, 20_000, prec, 300, 30, seed=1, init=init, model=model)
    run.propagate(300, 0.01, 30)
    sums = run.sums()
    for k in (8, 9, 14, 15):  # adiabatic populations (real, imaginary)
        assert np.all(sums[:, k] == sums[0, k])


def test_pure_dephasing_closed_form_fp32(q):
    model = pins._dephasing_model()
    init = pins._plus_init(model, beta=2.0)
    n, steps, stride, dt = 1 << 22, 400, 40, 0.01
    m, run = _gpu_run(q, None, n, q.PREC_FP32_BULK, steps, stride, seed=8, init=init, model=model)
    run.propagate(steps, dt, stride)
    obs = run.observables()
    disc, _ = pins._dephasing_closed_form(model, init, dt, np.arange(0, steps + 1, stride), 5.0)
    r01 = obs[:, 2] + 1j * obs[:, 3]
    se = obs[:, 16 + 2] + obs[:, 16 + 3]
    assert np.all(np.abs(r01 - 0.5 * disc) < 3 * se + 1e-6)
    assert np.abs(r01 - 0.5 * disc).max() < 1e-3


# ---------------------------------------------------------------- edges --
def test_step_mismatch_is_flagged_and_nothing_moves(q):
    cfg = wl.config(1)
    for prec in (q.PREC_FP64, q.PREC_FP32_BULK):
        m, run = _gpu_run(q, cfg, 300, prec, 100, 10)
        before = run.state()
        q.propagate(m, run.ens, run.ens_buf, 5, 10, 0.01, 10, run.obs_buf, run.n_out)
        st = run.status()
        assert st["flags"] & q.FLAG_STEP_MISMATCH
        assert st["step"] == 0
        after = run.state()
        assert np.array_equal(before["R"], after["R"])


def test_spin_boson_form_needs_b0_above_the_degeneracy_threshold(q):
    """A spin-boson model whose |b0| cannot keep r^2 = a^2 + b0^2 above the FP32
    degeneracy threshold runs the general two-state form, which tests for
    degeneracy: walkers held at a(R) = 0 (eps = 0, R0 = P0 = 0, no Wigner spread,
    so the mean force stays zero) count a degenerate step each step.  With b0
    large enough the spin-boson form runs and no step is degenerate."""
    for delta, expect in ((1e-7, True), (0.5, False)):
        model = wl.spin_boson(0.0, delta, np.array([1.0]), np.array([0.3]))
        init = {"rho_el0": np.diag([1.0, 0.0]), "R0": np.zeros(1), "P0": np.zeros(1),
                "beta": math.inf, "wigner": 0}
        n, steps = 1000, 40
        m, run = _gpu_run(q, None, n, q.PREC_FP32_BULK, steps, 10, init=init, model=model)
        run.propagate(steps, 0.01, 10)
        st = run.status()
        assert bool(st["flags"] & q.FLAG_DEGENERATE) == expect, delta
        assert st["n_degenerate"] == (n * steps if expect else 0), (delta, st)
        assert np.all(run.state()["R"] == 0.0)


def test_device_finalisation_matches_host_reduction(q):
    """qcl_finalize_observables writes the same rows as qcl_reduce_observables,
    on the device and without synchronising."""
    import torch

    cfg = wl.config(1)
    for prec in (q.PREC_FP64, q.PREC_FP32_BULK):
        m, run = _gpu_run(q, cfg, 3000, prec, 100, 10)
        run.propagate(100, cfg["dt"], 10)
        host = run.observables()
        dev = torch.full(host.shape, float("nan"), dtype=torch.float64, device="cuda")
        run.observables_device(dev)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), host)


def test_zero_steps_writes_only_initial_row(q):
    cfg = wl.config(1)
    for prec in (q.PREC_FP64, q.PREC_FP32_BULK):
        m, run = _gpu_run(q, cfg, 500, prec, 10, 10)
        run.obs_buf.zero_()
        run.propagate(0, 0.01, 10)
        sums = run.sums()
        assert np.all(sums[1] == 0) and sums[0, 16:].sum() > 0
        obs = run.observables()
        assert abs(obs[0, 32] - 1.0) < 0.1


def test_buffer_and_argument_errors(q):
    cfg = wl.config(1)
    m, run = _gpu_run(q, cfg, 300, q.PREC_FP32_BULK, 100, 10)
    with pytest.raises(q.QclError) as e:
        q.propagate(m, run.ens, run.ens_buf[: 1024], 0, 10, 0.01, 10, run.obs_buf, run.n_out)
    assert e.value.status == 3
    with pytest.raises(q.QclError) as e:
        q.propagate(m, run.ens, run.ens_buf, 0, 200, 0.01, 10, run.obs_buf, run.n_out)
    assert e.value.status == 1
    with pytest.raises(q.QclError) as e:
        q.propagate(m, run.ens, run.ens_buf, 0, 10, -0.01, 10, run.obs_buf, run.n_out)
    assert e.value.status == 1
    big = dict(cfg["model"])
    with pytest.raises(q.QclError) as e:
        q.Model(dict(big, E=np.array([[0.0, 1.0], [2.0, 0.0]])))
    assert e.value.status == 1


# ------------------------------------------------ full-size launch config --
def test_full_size_config2_sampled_walkers_and_invariants(q):
    """The launch configuration the benchmark times (1e7 walkers, 2000 steps,
    outputs every 10): sampled walkers checked one by one against the oracle at
    the start and after the first 50 steps (the FP32 walker's initial state
    advanced by the oracle: same decisions, R and P within 1e-5), and the
    ensemble invariants (trace, Hermitian partner) within 4 SE at every output
    time the estimator resolves (SE < 1e-2)."""
    cfg = wl.config(2)
    n, steps, stride = cfg["n_traj"], cfg["n_steps"], cfg["out_stride"]
    m, run = _gpu_run(q, cfg, n, q.PREC_FP32_BULK, steps, stride, seed=cfg["seed"])
    s0 = run.state()
    idx = np.unique(np.concatenate([np.linspace(0, n - 1, 200).astype(np.int64), [n - 1, n - 2]]))
    om = oracle.OracleModel(cfg["model"])
    oi = oracle.OracleInit(om, cfg["init"])
    for i in idx:
        ref = oracle.sample(om, oi, cfg["seed"], int(i), 1)
        assert np.allclose(s0["R"][i], ref.R[0], rtol=1e-5, atol=1e-6)
        assert (s0["alpha"][i], s0["beta"][i]) == (ref.alpha[0], ref.beta[0])
    # the sampled walkers' FP32 initial states, advanced 50 steps by the oracle
    seg = 50
    st = oracle.State(om, len(idx))
    st.R[:] = s0["R"][idx]
    st.P[:] = s0["P"][idx]
    st.m[:] = (s0["m"][idx].astype(np.float64) + s0["m_lo"][idx]) * np.ldexp(1.0, s0["m_exp"][idx])
    st.phi[:] = s0["phi"][idx].astype(np.float64) + s0["phi_lo"][idx]
    st.alpha[:] = s0["alpha"][idx]
    st.beta[:] = s0["beta"][idx]
    for k, i in enumerate(idx):
        one = oracle.State(om, 1)
        for key in ("R", "P", "m", "phi", "alpha", "beta"):
            getattr(one, key)[:] = getattr(st, key)[k:k + 1]
        oracle.advance(om, one, cfg["seed"], int(i), 0, seg, cfg["dt"])
        for key in ("R", "P", "m", "phi", "alpha", "beta"):
            getattr(st, key)[k] = getattr(one, key)[0]
    run.propagate(seg, cfg["dt"], stride)
    s1 = run.state()
    same = (s1["alpha"][idx] == st.alpha) & (s1["beta"][idx] == st.beta)
    assert same.all()
    for key, r in (("R", st.R), ("P", st.P)):
        scale = np.maximum(np.abs(r), np.abs(r).mean(axis=0, keepdims=True))
        assert (np.abs(s1[key][idx] - r) / scale).max() < 1e-5, key
    mw = (s1["m"][idx].astype(np.float64) + s1["m_lo"][idx]) * np.ldexp(1.0, s1["m_exp"][idx])
    assert np.median(np.abs(mw - st.m) / np.abs(st.m)) < 1e-6
    # the rest of the run, then the invariants where the estimator resolves
    run.propagate(steps - seg, cfg["dt"], stride)
    obs = run.observables()
    res = obs[:, 16 + 14] < 1e-2
    assert res.sum() >= 10
    tr, tr_se = obs[res, 32], obs[res, 16] + obs[res, 16 + 6]
    assert np.all(np.abs(tr - 1.0) < 4 * tr_se + 1e-9)
    d_re = obs[res, 2] - obs[res, 4]
    d_im = obs[res, 3] + obs[res, 5]
    assert np.all(np.abs(d_re) < 4 * (obs[res, 18] + obs[res, 20]) + 1e-12)
    assert np.all(np.abs(d_im) < 4 * (obs[res, 19] + obs[res, 21]) + 1e-12)
    assert np.all(np.isfinite(obs[:, :32]))
    assert run.status()["flags"] == 0
