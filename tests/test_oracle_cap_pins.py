"""Pins of the oracle's capped-probability branch (R4 of the transition rule:
p_e = min(kappa |A_e|, p_max) quantised to 24-bit thresholds; when they sum
above Tmax = floor(p_max 2^24) they are scaled down together, a hop to event e
multiplies the weight by A_e / p_hat_e and a stay by 1 / (1 - sum p_hat), both
over the scaled thresholds).

The cap changes only the sampling, never the expectation: whatever the
thresholds, a step's expected weight update is (1 + dt L) of Eq. 1 provided
every event keeps a nonzero threshold.  So the pins are

* the thresholds use the p_max budget and split it in proportion to the
  capped probabilities (the rule's definition stated as properties, checked
  against amplitudes that other pins tie to Eq. 1);
* walkers started at one phase-space point, in regimes where the cap binds at
  every branch point, reproduce the exact branch enumeration (each branch
  weighted by its amplitudes alone, no probabilities), in both
  representations, for two and four states;
* two plausible mistakes planted in a copy of the oracle (the stay factor from
  the sum before the cap, the hop factor from the probability before the cap)
  each fail that comparison.
"""
import math
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

from paper_2608_14544_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P24 = 2**24


def _dia3_model(p_max):
    E = np.array([[0.3, 0.25, 0.1], [0.25, -0.2, 0.15], [0.1, 0.15, 0.05]])
    K = np.zeros((1, 3, 3))
    K[0] = np.array([[0.4, 0.1, 0.0], [0.1, -0.3, 0.05], [0.0, 0.05, 0.1]])
    return {"name": "diabatic-3", "n_states": 3, "n_modes": 1, "hbar": 1.0,
            "mass": np.ones(1), "omega": np.ones(1), "E": E, "K": K, "hop_scale": 1.0,
            "p_max": p_max, "repr": "diabatic"}


def _cases():
    """(name, model, R0, P0, rho_el0, dt, steps) with the cap binding at every
    branch point of the enumeration (checked in the tests)."""
    out = []
    # two-state adiabatic, each event also above p_max on its own
    m = wl.spin_boson(0.0, 0.5, [1.0], [1.0])
    m["p_max"] = 0.05
    out.append(("adiabatic-2-capped", m, [0.1], [2.0], np.diag([1.0, 0.0]), 0.05, 5))
    # two-state adiabatic, each event below p_max, their sum above (rescale only)
    m = wl.spin_boson(0.0, 0.5, [1.0], [1.0])
    m["p_max"] = 0.05
    out.append(("adiabatic-2-rescaled", m, [0.1], [2.0], np.diag([1.0, 0.0]), 0.02, 6))
    # four states, unequal events (the proportional integer rescale matters)
    m = wl.random_lvc4(7, n_modes=2)
    m["p_max"] = 0.05
    rho = np.zeros((4, 4))
    rho[1, 1] = 1.0
    out.append(("adiabatic-4", m, [0.3, -0.2], [1.5, 1.0], rho, 0.05, 4))
    # two-state diabatic
    m = wl.spin_boson(0.3, 0.5, [1.0], [1.0])
    m["repr"] = "diabatic"
    m["p_max"] = 0.04
    out.append(("diabatic-2", m, [0.4], [1.5], np.array([[0.7, 0.3], [0.3, 0.3]]), 0.05, 6))
    # three-state diabatic
    rho = np.array([[0.6, 0.2, 0.1], [0.2, 0.3, 0.05], [0.1, 0.05, 0.1]])
    out.append(("diabatic-3", _dia3_model(0.02), [0.3], [1.0], rho, 0.1, 4))
    return out


CASES = {c[0]: c for c in _cases()}


def _events(O, om, model, R1, P1, a, b, dt):
    """Amplitudes (complex for the diabatic representation) and thresholds."""
    if model.get("repr") == "diabatic":
        ta, tb, c, dq, T = O.events_dia(om, R1, a, b, dt)
        return ta, tb, c * (1j ** dq), np.abs(c), T
    e1, U1, _ = O.adiabatic(om, R1)
    ta, tb, A, T = O.events(om, P1, e1, U1, a, b, dt)
    return ta, tb, A.astype(complex), np.abs(A), T


def _enumerate(O, model, R0, P0, rho, dt, k):
    """Exact expectation of every observable after 0..k steps from one point:
    each branch (stay, or an event with a nonzero threshold) carries its own
    trajectory and the product of its amplitudes.  Models with more than two
    adiabatic states carry each branch's eigenvectors by parallel transport, as
    the walkers do (the amplitudes and the rotated observables depend on that
    gauge, their products along a branch do not).  Also returns, over all
    branch points, the fraction where the pre-cap probabilities exceed p_max."""
    om = O.OracleModel(model)
    ns = model["n_states"]
    nq = 4 * ns * ns
    dia = model.get("repr") == "diabatic"
    carry = ns > 2 and not dia
    R0, P0 = np.asarray(R0, float), np.asarray(P0, float)
    _, U0, _ = O.adiabatic(om, R0)
    rho_w = rho if dia else U0.T @ rho @ U0
    T0 = np.floor(np.abs(rho_w) / np.abs(rho_w).sum() * P24)
    br = [(R0.copy(), P0.copy(), 0.0, a, b, complex(rho_w[a, b]), U0.copy())
          for a in range(ns) for b in range(ns) if rho_w[a, b] != 0 and T0[a, b] > 0]

    def obs(R, a, b, w, phi, U):
        Uo = U if carry else O.adiabatic(om, R)[1]
        z = w * np.exp(-1j * phi)
        q = np.zeros(nq)
        own, other = (0, 2 * ns * ns) if dia else (2 * ns * ns, 0)
        q[own + 2 * (a * ns + b)] = z.real
        q[own + 2 * (a * ns + b) + 1] = z.imag
        for i in range(ns):
            for j in range(ns):
                # adiabatic walker -> diabatic rho_ij = z U_ia U_jb; diabatic
                # walker -> adiabatic rho_ij = z U_ai U_bj
                v = z * (Uo[a, i] * Uo[b, j] if dia else Uo[i, a] * Uo[j, b])
                q[other + 2 * (i * ns + j)] = v.real
                q[other + 2 * (i * ns + j) + 1] = v.imag
        return q

    rows = np.zeros((k + 1, nq))
    for R, P, phi, a, b, w, U in br:
        rows[0] += obs(R, a, b, w, phi, U)
    points = capped = 0
    for n in range(1, k + 1):
        nxt = []
        for R, P, phi, a, b, w, U in br:
            R1, P1, phi1, _ = O.step_deterministic(om, R, P, phi, a, b, U.copy(), dt)
            if dia:
                ta, tb, c, dq, T = O.events_dia(om, R1, a, b, dt)
                amp, mag, U1 = c * (1j ** dq), np.abs(c), U
            else:
                e1, U1, _ = O.adiabatic(om, R1, U if carry else None)
                ta, tb, A, T = O.events(om, P1, e1, U1, a, b, dt)
                amp, mag = A.astype(complex), np.abs(A)
            p = np.minimum(model["hop_scale"] * mag, model["p_max"])
            points += 1
            capped += np.floor(p * P24).sum() > math.floor(model["p_max"] * P24)
            nxt.append((R1, P1, phi1, a, b, w, U1))
            for t in range(len(T)):
                if T[t] > 0:
                    nxt.append((R1, P1, phi1, int(ta[t]), int(tb[t]), w * amp[t], U1))
        br = nxt
        for R, P, phi, a, b, w, U in br:
            rows[n] += obs(R, a, b, w, phi, U)
    return rows, capped / points


def _walker_z(O, model, R0, P0, rho, dt, k, n, seed=21):
    om = O.OracleModel(model)
    init = {"rho_el0": rho, "R0": np.asarray(R0, float), "P0": np.asarray(P0, float),
            "beta": math.inf, "wigner": 0}
    rows, _ = O.run(om, O.OracleInit(om, init), seed, 0, n, dt, k, 1)
    mean, se = O.finalize(rows, n)
    exact, frac = _enumerate(O, model, R0, P0, rho, dt, k)
    z = np.abs(mean - exact) / np.maximum(se, 1e-15)
    z[np.abs(mean - exact) < 1e-12] = 0.0
    return z, exact, frac


# ------------------------------------------------------------- thresholds --
@pytest.mark.parametrize("name", sorted(CASES))
def test_capped_thresholds_fill_the_budget_in_proportion(oracle_lib, name):
    _, model, R0, P0, rho, dt, _ = CASES[name]
    O = oracle_lib
    om = O.OracleModel(model)
    ns, n = model["n_states"], model["n_modes"]
    tmax = math.floor(model["p_max"] * P24)
    rng = np.random.default_rng(5)
    seen = 0
    for _ in range(40):
        R = np.asarray(R0) + 0.3 * rng.normal(size=n)
        P = np.asarray(P0) * rng.uniform(0.5, 1.5, size=n)
        a, b = (int(x) for x in rng.integers(0, ns, size=2))
        ta, tb, amp, mag, T = _events(O, om, model, R, P, a, b, dt)
        p = np.minimum(model["hop_scale"] * mag, model["p_max"])
        ne = len(T)
        assert ne == 2 * (ns - 1)
        T = T.astype(np.int64)
        assert T.sum() <= tmax
        if p.sum() <= model["p_max"] * (1 - 1e-9):
            continue  # below the cap: each threshold is its own probability
        seen += 1
        # the whole budget is used, up to the floor of each share
        assert T.sum() >= tmax - ne
        # shares in proportion to the capped probabilities
        share = tmax * p / p.sum()
        assert np.all(np.abs(T - share) <= ne + 1), (T, share)
        # equal events get exactly equal thresholds
        for i in range(ne):
            for j in range(ne):
                if p[i] == p[j]:
                    assert T[i] == T[j]
    assert seen >= 10


# -------------------------------------------------- enumeration in the cap --
@pytest.mark.parametrize("name", sorted(CASES))
def test_capped_walkers_match_branch_enumeration(oracle_lib, name):
    _, model, R0, P0, rho, dt, k = CASES[name]
    z, exact, frac = _walker_z(oracle_lib, model, R0, P0, rho, dt, k, 400_000)
    assert frac == 1.0, f"the cap binds at only {frac:.2f} of the branch points"
    assert z.max() < 4.5, z.max()
    # transitions fired: weight moved away from the initial populations
    assert np.abs(exact[k] - exact[0]).max() > 1e-2


# ----------------------------------------------------- planted mistakes --
_PRECAP = """
static double precap_sum(const orc_model* md, const double* amp, int ne) {
  double s = 0.0;
  for (int k = 0; k < ne; ++k) {
    double p = md->hop_scale * fabs(amp[k]);
    if (p > md->p_max) p = md->p_max;
    s += floor(p * P24);
  }
  return s / P24;
}
"""


def _mutant(src: str, kind: str) -> str:
    anchor = "static void full_step_dia("
    assert src.count(anchor) == 1
    src = src.replace(anchor, _PRECAP + anchor)
    if kind == "stay":
        old = "(double)tot / P24"
        assert src.count(old) == 2
        src = src.replace(old, "precap_sum(md, c, ne)", 1).replace(old, "precap_sum(md, A, ne)", 1)
    else:
        old = "double phat = (double)T[k] / P24;"
        assert src.count(old) == 2
        new = ("double phat = floor(fmin(md->hop_scale * fabs({x}[k]), md->p_max) * P24) / P24;")
        src = src.replace(old, new.format(x="c"), 1).replace(old, new.format(x="A"), 1)
    return src


_CHILD = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from tests import test_oracle_cap_pins as t
import oracle as O
name = {name!r}
_, model, R0, P0, rho, dt, k = t.CASES[name]
z, _, _ = t._walker_z(O, model, R0, P0, rho, dt, k, 200_000)
print("ZMAX", float(z.max()))
"""


@pytest.mark.parametrize("kind", ["stay", "hop"])
@pytest.mark.parametrize("name", ["adiabatic-2-capped", "adiabatic-4", "diabatic-2"])
def test_planted_cap_mistakes_fail_the_enumeration_pin(oracle_lib, tmp_path, kind, name):
    """A copy of the oracle with the stay factor (or the hop factor) taken from
    the probabilities before the cap is biased, and the enumeration pin sees it."""
    here = os.path.join(ROOT, "oracle")
    with open(os.path.join(here, "qcl_oracle.c")) as f:
        src = f.read()
    mdir = tmp_path / "oracle_mutant"
    mdir.mkdir()
    (mdir / "qcl_oracle.c").write_text(_mutant(src, kind))
    shutil.copy(os.path.join(here, "qcl_oracle.h"), mdir / "qcl_oracle.h")
    env = dict(os.environ, QCL_ORACLE_SRC=str(mdir / "qcl_oracle.c"),
               QCL_ORACLE_LIB=str(mdir / "liboracle_mutant.so"))
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT, name=name)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    zmax = float(r.stdout.split("ZMAX")[1])
    assert zmax > 8.0, f"planted {kind} mistake not detected on {name} (z = {zmax:.2f})"
