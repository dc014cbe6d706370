"""Pins of the oracle's trajectory-spawning scheme (the CPU code's scheme that
the paper's GPU version replaces): a fired transition test leaves the walker
in place and spawns a child at the target pair with weight m A_e / p_hat_e.

* Exact expectation: the family-summed ensemble mean matches exhaustive branch
  enumeration (the same expectation as the no-spawn scheme), adiabatic and
  diabatic.
* With no coupling nothing spawns and every row equals the no-spawn run's bits.
* Walker level: a family's first child is born exactly where the no-spawn
  walker with the same random stream makes its first hop, on the same (R, P,
  phi) and pair, with the no-spawn weight divided by that walker's accumulated
  stay factors.
* Standard error: the family-based SE matches the spread of the mean over
  independent replicas.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_14544_gb300 import workloads as wl
from tests.test_oracle_diabatic_pins import _enumerate_dia
from tests.test_oracle_pins import _dephasing_model, _enumerate, _plus_init


def _point_init(R0, P0, rho):
    return {"rho_el0": rho, "R0": np.asarray(R0, float), "P0": np.asarray(P0, float),
            "beta": math.inf, "wigner": 0}


@pytest.mark.parametrize("rep", ["adiabatic", "diabatic"])
def test_spawn_ensemble_matches_branch_enumeration(rep):
    model = wl.spin_boson(0.3 if rep == "diabatic" else 0.0, 0.5, [1.0], [1.0])
    model["repr"] = rep
    om = O.OracleModel(model)
    R0, P0 = np.array([0.4]), np.array([1.5])
    rho = np.array([[1.0, 0.0], [0.0, 0.0]]) if rep == "adiabatic" else \
        np.array([[0.7, 0.3], [0.3, 0.3]])
    init = _point_init(R0, P0, rho)
    dt, k, n0 = 0.05, 6, 200_000
    if rep == "adiabatic":
        exact = _enumerate(O, om, model, R0, P0, rho, dt, k)
    else:
        exact = _enumerate_dia(om, model, R0, P0, rho, dt, k)
    rows, n_live = O.run_spawn(om, O.OracleInit(om, init), 21, 0, n0, 4 * n0, dt, k, 1)
    mean, se = O.finalize(rows, n0)
    z = np.abs(mean - exact) / np.maximum(se, 1e-15)
    assert np.all((z < 4.5) | (np.abs(mean - exact) < 1e-12)), z.max()
    assert n_live[-1] > n0 * 1.05  # children were spawned
    assert np.all(np.diff(n_live) >= 0)


def test_no_coupling_spawns_nothing_and_matches_no_spawn_bits():
    model = _dephasing_model()
    init = _plus_init(model, beta=2.0)
    om = O.OracleModel(model)
    oi = O.OracleInit(om, init)
    rows_s, n_live = O.run_spawn(om, oi, 5, 0, 3000, 3000, 0.01, 200, 20)
    rows, _ = O.run(om, oi, 5, 0, 3000, 0.01, 200, 20)
    assert np.all(n_live == 3000)
    assert np.array_equal(rows_s, rows)


def test_first_child_is_born_at_the_no_spawn_walkers_first_hop():
    cfg = wl.config(1)
    om = O.OracleModel(cfg["model"])
    oi = O.OracleInit(om, cfg["init"])
    n0, steps, dt, seed = 64, 300, cfg["dt"], 3
    ns_st = O.sample(om, oi, seed, 0, n0)
    sp = O.spawn_sample(om, oi, seed, 0, n0, 200_000)
    first_hop = {}
    m_before = ns_st.m.copy()
    for s in range(steps):
        prev = (ns_st.alpha.copy(), ns_st.beta.copy(), ns_st.m.copy())
        O.advance(om, ns_st, seed, 0, s, 1, dt)
        n_before = sp.n_live
        fam_before = sp.family[:n_before].copy()
        assert O.spawn_advance(om, sp, seed, s, 1, dt) == 0
        live = sp.live()
        for i in range(n0):
            if i in first_hop:
                continue
            hopped = (ns_st.alpha[i], ns_st.beta[i]) != (prev[0][i], prev[1][i])
            members = np.where(live["family"] == i)[0]
            born = len(members) > np.sum(fam_before == i)
            assert hopped == born, (s, i)
            if hopped:
                first_hop[i] = s
                root, child = members[0], members[1]
                assert live["id"][root] == i and live["id"][child] >= np.uint64(1 << 63)
                assert (live["alpha"][child], live["beta"][child]) == (ns_st.alpha[i], ns_st.beta[i])
                for key, ref in (("R", ns_st.R[i]), ("P", ns_st.P[i])):
                    assert np.allclose(live[key][child], ref, rtol=1e-13, atol=1e-13)
                assert live["phi"][child] == pytest.approx(ns_st.phi[i], rel=1e-13, abs=1e-13)
                # no-spawn weight = child weight x (stay factors accumulated so far)
                stay = prev[2][i] / live["m"][root]
                assert ns_st.m[i] == pytest.approx(live["m"][child] * stay, rel=1e-12)
    assert len(first_hop) > 10
    # families stay contiguous and in order
    fam = sp.live()["family"]
    assert np.all(np.diff(fam) >= 0)


def test_family_standard_error_matches_replica_spread():
    cfg = wl.config(1)
    om = O.OracleModel(cfg["model"])
    oi = O.OracleInit(om, cfg["init"])
    n0, steps, stride, reps = 400, 200, 50, 40
    means, ses = [], []
    for r in range(reps):
        rows, _ = O.run_spawn(om, oi, 100 + r, 0, n0, 50 * n0, cfg["dt"], steps, stride)
        mean, se = O.finalize(rows, n0)
        means.append(mean[-1])
        ses.append(se[-1])
    means, ses = np.array(means), np.array(ses)
    k = [0, 2, 14]  # rho_00 (diabatic), Re rho_01, adiabatic upper population
    spread = means[:, k].std(axis=0, ddof=1)
    reported = np.sqrt((ses[:, k] ** 2).mean(axis=0))
    # the standard deviation of a 40-sample estimate is about 11 %
    assert np.all(np.abs(spread / reported - 1.0) < 0.4), spread / reported


def test_observation_sums_families_before_squaring():
    cfg = wl.config(1)
    om = O.OracleModel(cfg["model"])
    oi = O.OracleInit(om, cfg["init"])
    n0 = 300
    sp = O.spawn_sample(om, oi, 8, 0, n0, 100_000)
    assert O.spawn_advance(om, sp, 8, 0, 250, cfg["dt"]) == 0
    assert sp.n_live > 2 * n0
    row = O.spawn_observe(om, sp)
    # per-walker contributions of the live walkers, grouped by family in numpy
    live = O.State(om, sp.n_live)
    for k in ("R", "P", "m", "phi", "alpha", "beta", "q"):
        getattr(live, k)[:] = getattr(sp, k)[:sp.n_live]
    qw = O.contrib(om, live)
    X = np.zeros((n0, qw.shape[1]))
    np.add.at(X, sp.family[:sp.n_live], qw)
    nq = qw.shape[1]
    assert np.allclose(row[:nq], X.sum(axis=0), rtol=1e-12, atol=1e-12)
    assert np.allclose(row[nq:], (X ** 2).sum(axis=0), rtol=1e-12, atol=1e-12)
    # the grouping matters: per-walker squares differ from family squares
    assert not np.allclose(row[nq:], (qw ** 2).sum(axis=0), rtol=1e-3)


def test_three_state_diabatic_spawn_ensemble_matches_branch_enumeration():
    """Spawning for three states (four events per step besides the stay, each
    child with its event's quarter turns): the family-summed mean against the
    exact enumeration of every branch."""
    E = np.diag([0.0, 0.3, 0.7]) + 0.1 * (np.ones((3, 3)) - np.eye(3))
    K = np.zeros((2, 3, 3))
    K[0] = np.array([[0.4, 0.2, 0.0], [0.2, -0.3, 0.15], [0.0, 0.15, 0.1]])
    K[1] = np.array([[-0.2, 0.05, 0.25], [0.05, 0.3, -0.1], [0.25, -0.1, 0.0]])
    model = wl._model(E, K, np.ones(2), np.array([1.0, 1.3]), name="lvc3-spawn-pin")
    model["repr"] = "diabatic"
    om = O.OracleModel(model)
    R0, P0 = np.array([0.3, -0.5]), np.array([1.2, 0.8])
    rho = np.array([[0.6, 0.2, 0.0], [0.2, 0.3, 0.1], [0.0, 0.1, 0.1]])
    dt, k, n0 = 0.1, 4, 200_000
    exact = _enumerate_dia(om, model, R0, P0, rho, dt, k)
    rows, n_live = O.run_spawn(om, O.OracleInit(om, _point_init(R0, P0, rho)), 31, 0, n0,
                               8 * n0, dt, k, 1)
    mean, se = O.finalize(rows, n0)
    z = np.abs(mean - exact) / np.maximum(se, 1e-15)
    assert np.all((z < 4.5) | (np.abs(mean - exact) < 1e-12)), z.max()
    assert n_live[-1] > n0 * 1.05
