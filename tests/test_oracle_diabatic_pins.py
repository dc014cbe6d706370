"""Pins of the oracle's diabatic representation (the coupling enters as the
off-diagonal potential, amplitudes -i V dt/hbar and +i V dt/hbar, weights
carried with a quarter-turn count).

* Frozen nuclei (K = 0): the electronic equation is the Liouville-von Neumann
  equation with the constant Hamiltonian E, solved exactly by exp(-iEt/hbar).
  The estimator's expectation obeys a linear recursion (exact diagonal phase,
  first-order off-diagonal transfer) that converges to that solution; the
  walker ensemble must reproduce the recursion within its standard error.
* Delta = 0 at any eps (including the crossing regime the adiabatic test
  cannot use): no transition fires and the coherence is the Gaussian
  characteristic function of the linear phase functional (closed form).
* Branch enumeration with nuclear coupling: every stay/hop branch carries its
  own trajectory and complex weight; the ensemble mean must match their sum.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import oracle as O
from paper_2608_14544_gb300 import workloads as wl
from tests.test_oracle_pins import _dephasing_closed_form, _dephasing_model, _plus_init


def _frozen_model(E):
    E = np.asarray(E, dtype=np.float64)
    ns = E.shape[0]
    return {"name": "frozen", "n_states": ns, "n_modes": 1, "hbar": 1.0,
            "mass": np.ones(1), "omega": np.ones(1), "E": E,
            "K": np.zeros((1, ns, ns)), "hop_scale": 1.0, "p_max": 0.5,
            "repr": "diabatic"}


def _recursion(E, rho0, dt, n_steps, hbar=1.0):
    """Expectation of the diabatic estimator: per step the exact diagonal phase
    D = Phi o rho (Phi_ab = exp(-i (E_aa - E_bb) dt / hbar)), then the
    off-diagonal transfer D - i C D + i D C with C = offdiag(E) dt / hbar."""
    d = np.diag(E)
    Phi = np.exp(-1j * (d[:, None] - d[None, :]) * dt / hbar)
    C = (E - np.diag(d)) * dt / hbar
    rho = rho0.astype(complex)
    out = [rho.copy()]
    for _ in range(n_steps):
        D = Phi * rho
        rho = D - 1j * (C @ D) + 1j * (D @ C)
        out.append(rho.copy())
    return np.array(out)


E3 = np.array([[0.3, 0.25, 0.1], [0.25, -0.2, 0.15], [0.1, 0.15, 0.05]])
RHO3 = np.array([[0.6, 0.2, 0.1], [0.2, 0.3, 0.05], [0.1, 0.05, 0.1]])


def test_expectation_recursion_converges_to_liouville_von_neumann():
    t_end = 4.0
    errs = []
    for dt in (0.02, 0.01, 0.005):
        n = int(round(t_end / dt))
        rec = _recursion(E3, RHO3, dt, n)[-1]
        U = expm(-1j * E3 * t_end)
        exact = U @ RHO3 @ U.conj().T
        errs.append(np.abs(rec - exact).max())
    # first order in dt, and small
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.15)
    assert errs[1] / errs[2] == pytest.approx(2.0, rel=0.15)
    assert errs[2] < 5e-3


def test_frozen_nuclei_ensemble_matches_recursion():
    model = _frozen_model(E3)
    om = O.OracleModel(model)
    init = {"rho_el0": RHO3, "R0": np.zeros(1), "P0": np.zeros(1), "beta": math.inf, "wigner": 1}
    oi = O.OracleInit(om, init)
    dt, n_steps, stride, n = 0.05, 80, 10, 100_000
    rows, _ = O.run(om, oi, 17, 0, n, dt, n_steps, stride)
    mean, se = O.finalize(rows, n)
    rec = _recursion(E3, RHO3, dt, n_steps)[::stride]
    ns = 3
    got = mean[:, 0:2 * ns * ns:2] + 1j * mean[:, 1:2 * ns * ns:2]
    sig = se[:, 0:2 * ns * ns:2] + 1j * se[:, 1:2 * ns * ns:2]
    want = rec.reshape(len(rec), ns * ns)
    z_re = np.abs(got.real - want.real) / np.maximum(sig.real, 1e-15)
    z_im = np.abs(got.imag - want.imag) / np.maximum(sig.imag, 1e-15)
    assert np.all((z_re < 4.5) | (np.abs(got.real - want.real) < 1e-12)), z_re.max()
    assert np.all((z_im < 4.5) | (np.abs(got.imag - want.imag) < 1e-12)), z_im.max()
    # the electronic dynamics really moved: at some output the populations and
    # coherences have changed by many standard errors, and imaginary parts appear
    moved = np.abs(want - want[0]).max(axis=1) / np.maximum(sig.real.max(axis=1), 1e-15)
    assert moved.max() > 10, moved
    assert np.abs(want[-1].imag).max() > 0.05
    # adiabatic block = U^T rho_dia U with the constant eigenvectors (populations
    # are gauge-free)
    w, V = np.linalg.eigh(E3)
    got_ad = mean[:, 2 * ns * ns::2] + 1j * mean[:, 2 * ns * ns + 1::2]
    for k in range(len(rec)):
        ad = V.T @ got[k].reshape(ns, ns) @ V
        assert np.allclose(np.diag(ad), np.diag(got_ad[k].reshape(ns, ns)), atol=1e-12)


def test_frozen_nuclei_diabatic_agrees_with_exact_adiabatic():
    """With K = 0 the adiabatic representation has no coupling (d = 0) and is
    exact for the diagonalised problem; the diabatic walkers estimate the same
    adiabatic populations."""
    E2 = np.array([[0.2, 0.3], [0.3, -0.2]])
    rho = np.array([[1.0, 0.0], [0.0, 0.0]])
    dt, n_steps, stride, n = 0.02, 200, 20, 60_000
    out = {}
    for rep in ("adiabatic", "diabatic"):
        model = _frozen_model(E2)
        model["repr"] = rep
        om = O.OracleModel(model)
        init = {"rho_el0": rho, "R0": np.zeros(1), "P0": np.zeros(1), "beta": math.inf,
                "wigner": 0}
        rows, _ = O.run(om, O.OracleInit(om, init), 3, 0, n, dt, n_steps, stride)
        out[rep] = O.finalize(rows, n)
    ma, sa = out["adiabatic"]
    md, sd = out["diabatic"]
    for k in (8, 14):  # adiabatic populations rho_00, rho_11 (both estimators are noisy)
        assert np.all(np.abs(md[:, k] - ma[:, k]) < 4.5 * np.hypot(sd[:, k], sa[:, k]) + 1e-12)
    # the adiabatic run is deterministic here: every walker keeps its pair
    assert np.abs(ma[:, 8] - ma[0, 8]).max() < 1e-12
    # the diabatic population oscillates (Rabi): the comparison is not trivial
    assert np.abs(md[:, 0] - md[0, 0]).max() > 0.2


@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_diabatic_pure_dephasing_at_any_eps(eps):
    model = _dephasing_model(eps=eps)
    model["repr"] = "diabatic"
    init = _plus_init(model, beta=2.0)
    om = O.OracleModel(model)
    oi = O.OracleInit(om, init)
    dt, n_steps, stride, n_traj = 0.01, 400, 40, 40_000
    rows, _ = O.run(om, oi, 5, 0, n_traj, dt, n_steps, stride)
    mean, se = O.finalize(rows, n_traj)
    steps = np.arange(0, n_steps + 1, stride)
    disc, exact = _dephasing_closed_form(model, init, dt, steps, eps)
    assert np.abs(disc - exact).max() < 1e-3
    r01 = mean[:, 2] + 1j * mean[:, 3]
    s01 = se[:, 2] + 1j * se[:, 3]
    assert np.all(np.abs(r01.real - 0.5 * disc.real) < 4 * s01.real + 1e-12)
    assert np.all(np.abs(r01.imag - 0.5 * disc.imag) < 4 * s01.imag + 1e-12)
    # no transition can fire: the diabatic populations are exactly constant
    assert np.all(rows[:, 0] == rows[0, 0]) and np.all(rows[:, 6] == rows[0, 6])
    assert abs(disc[-1]) < 0.9
    # walker level: pairs, weights and quarter turns never change
    st = O.sample(om, oi, 5, 0, 256)
    s0 = st.copy()
    O.advance(om, st, 5, 0, 0, 200, dt)
    assert np.array_equal(st.alpha, s0.alpha) and np.array_equal(st.beta, s0.beta)
    assert np.array_equal(st.m, s0.m) and np.all(st.q == 0)


def _lvc8(n, seed):
    rng = np.random.default_rng(seed)
    E = np.diag(0.4 * np.arange(8)) + 0.04 * (np.ones((8, 8)) - np.eye(8))
    K = np.zeros((n, 8, 8))
    for j in range(n):
        a = rng.normal(size=(8, 8)) * 0.12 * np.sqrt(6.0 / n)
        K[j] = 0.5 * (a + a.T)
    return wl._model(E, K, np.ones(n), rng.uniform(0.6, 1.5, size=n), name=f"lvc8x{n}")


# (four states with 6 and 40 modes, eight states with 12: the sizes the FP32
# kernels are compared at)
@pytest.mark.parametrize("make", [lambda: wl.random_lvc4(3), lambda: wl.random_lvc4(3, 40),
                                  lambda: _lvc8(12, 4)])
def test_diabatic_events_follow_the_off_diagonal_potential(make):
    model = make()
    model["repr"] = "diabatic"
    om = O.OracleModel(model)
    rng = np.random.default_rng(2)
    dt, ns = 0.05, model["n_states"]
    for _ in range(20):
        R = rng.normal(size=model["n_modes"])
        W = model["E"] + np.einsum("j,jab->ab", R, model["K"])
        a, b = rng.integers(0, ns, size=2)
        ta, tb, c, dq, T = O.events_dia(om, R, int(a), int(b), dt)
        k = 0
        for g in range(ns):
            if g == a:
                continue
            assert (ta[k], tb[k], dq[k]) == (g, b, 3)
            assert c[k] == pytest.approx(W[g, a] * dt / model["hbar"], rel=1e-13, abs=1e-15)
            k += 1
        for g in range(ns):
            if g == b:
                continue
            assert (ta[k], tb[k], dq[k]) == (a, g, 1)
            assert c[k] == pytest.approx(W[b, g] * dt / model["hbar"], rel=1e-13, abs=1e-15)
            k += 1
        # thresholds: never above the p_max budget, monotone in |c| (the capped
        # split itself is pinned by the branch enumeration in the capped regime)
        assert int(T.astype(np.int64).sum()) <= int(np.floor(model["p_max"] * 2**24))
        order = np.argsort(np.abs(c), kind="stable")
        assert np.all(np.diff(T[order].astype(np.int64)) >= 0)


def _enumerate_dia(om, model, R0, P0, rho_el0, dt, k):
    """Exact expectation after 0..k steps from one phase-space point: every
    branch (stay, or each event with T > 0) with its own trajectory and complex
    weight (product of the amplitudes c i^dq)."""
    ns = model["n_states"]
    nq = 4 * ns * ns
    tot = np.abs(rho_el0).sum()
    T0 = np.floor(np.abs(rho_el0) / tot * 2**24)
    branches = [(R0.copy(), P0.copy(), 0.0, a, b, complex(rho_el0[a, b]))
                for a in range(ns) for b in range(ns) if rho_el0[a, b] != 0 and T0[a, b] > 0]

    def obs(R, a, b, w, phi):
        _, Uo, _ = O.adiabatic(om, R)
        z = w * np.exp(-1j * phi)
        q = np.zeros(nq)
        q[2 * (a * ns + b)] = z.real
        q[2 * (a * ns + b) + 1] = z.imag
        for kk in range(ns):
            for ll in range(ns):
                v = z * Uo[a, kk] * Uo[b, ll]
                q[2 * ns * ns + 2 * (kk * ns + ll)] = v.real
                q[2 * ns * ns + 2 * (kk * ns + ll) + 1] = v.imag
        return q

    rows = np.zeros((k + 1, nq))
    for br in branches:
        rows[0] += obs(br[0], br[3], br[4], br[5], br[2])
    for n in range(1, k + 1):
        nxt = []
        for R, P, phi, a, b, w in branches:
            R1, P1, phi1, _ = O.step_deterministic(om, R, P, phi, a, b, None, dt)
            ta, tb, c, dq, T = O.events_dia(om, R1, a, b, dt)
            nxt.append((R1, P1, phi1, a, b, w))
            for t in range(len(c)):
                if T[t] > 0:
                    nxt.append((R1, P1, phi1, int(ta[t]), int(tb[t]), w * c[t] * 1j ** int(dq[t])))
        branches = nxt
        for R, P, phi, a, b, w in branches:
            rows[n] += obs(R, a, b, w, phi)
    return rows


def test_diabatic_walkers_match_branch_enumeration():
    model = wl.spin_boson(0.3, 0.5, [1.0], [1.0])
    model["repr"] = "diabatic"
    om = O.OracleModel(model)
    R0, P0 = np.array([0.4]), np.array([1.5])
    rho = np.array([[0.7, 0.3], [0.3, 0.3]])
    init = {"rho_el0": rho, "R0": R0, "P0": P0, "beta": math.inf, "wigner": 0}
    oi = O.OracleInit(om, init)
    dt, k, n = 0.05, 6, 400_000
    exact = _enumerate_dia(om, model, R0, P0, rho, dt, k)
    rows, _ = O.run(om, oi, 21, 0, n, dt, k, 1)
    mean, se = O.finalize(rows, n)
    z = np.abs(mean - exact) / np.maximum(se, 1e-15)
    assert np.all((z < 4.5) | (np.abs(mean - exact) < 1e-12)), z.max()
    # transitions fired: the populations moved and imaginary parts appeared
    assert abs(exact[k, 0] - exact[0, 0]) > 1e-3
    assert np.abs(exact[k, 1::2]).max() > 1e-3


def test_diabatic_three_state_walkers_match_branch_enumeration():
    """The same enumeration for three states with nuclear coupling in every
    K_j: four events per step (two per index) besides the stay, each with its
    own quarter turns, and the adiabatic block rotated by the eigenvectors at
    each branch's R."""
    E = np.diag([0.0, 0.3, 0.7]) + 0.1 * (np.ones((3, 3)) - np.eye(3))
    K = np.zeros((2, 3, 3))
    K[0] = np.array([[0.4, 0.2, 0.0], [0.2, -0.3, 0.15], [0.0, 0.15, 0.1]])
    K[1] = np.array([[-0.2, 0.05, 0.25], [0.05, 0.3, -0.1], [0.25, -0.1, 0.0]])
    model = wl._model(E, K, np.ones(2), np.array([1.0, 1.3]), name="lvc3-dia-pin")
    model["repr"] = "diabatic"
    om = O.OracleModel(model)
    R0, P0 = np.array([0.3, -0.5]), np.array([1.2, 0.8])
    rho = np.array([[0.6, 0.2, 0.0], [0.2, 0.3, 0.1], [0.0, 0.1, 0.1]])
    init = {"rho_el0": rho, "R0": R0, "P0": P0, "beta": math.inf, "wigner": 0}
    dt, k, n = 0.1, 4, 400_000
    exact = _enumerate_dia(om, model, R0, P0, rho, dt, k)
    rows, _ = O.run(om, O.OracleInit(om, init), 23, 0, n, dt, k, 1)
    mean, se = O.finalize(rows, n)
    z = np.abs(mean - exact) / np.maximum(se, 1e-15)
    assert np.all((z < 4.5) | (np.abs(mean - exact) < 1e-12)), z.max()
    # transitions fired into every state and the coherences turned complex
    assert abs(exact[k, 2 * (2 * 3 + 2)] - exact[0, 2 * (2 * 3 + 2)]) > 1e-3
    assert np.abs(exact[k, 1:18:2]).max() > 1e-3
