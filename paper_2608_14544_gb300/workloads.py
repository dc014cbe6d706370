"""Seeded synthetic workloads: model Hamiltonians, initial conditions and run
parameters for the spin-boson and vibronic systems of the paper (Sec. II C).

This module only builds input parameters.  It holds none of the propagation
arithmetic and is shared by the CUDA path's tests and benchmark and by the
oracle-side tests.  The paper cites, but does not print, its model parameters,
so the values below are stated readings:

* spin-boson: W(R) = eps sigma_z + Delta sigma_x + sum_j c_j R_j sigma_z, with the
  bath centred at the minimum of the initially occupied diabatic surface,
  R0_j = -c_j / (M_j w_j^2);
* ohmic bath J(w) = (pi/2) xi w exp(-w/wc), discretised with equal density of
  modes: w_j = -wc ln(1 - j/(N+1)), c_j = w_j sqrt(xi wc / (N+1)), M_j = 1;
* the two-state three-mode vibronic model with a conical intersection is a
  declared synthetic linear vibronic-coupling model (eV / fs units), since the
  pyrazine parameters are not given in the paper;
* the random four-state model draws its parameters from numpy's seeded
  generator (seed = request id).
"""
from __future__ import annotations

import math

import numpy as np

HBAR_EV_FS = 0.6582119569  # eV fs

SX = np.array([[0.0, 1.0], [1.0, 0.0]])
SZ = np.array([[1.0, 0.0], [0.0, -1.0]])


def _model(E, K, mass, omega, hbar=1.0, hop_scale=1.0, p_max=0.5, name=""):
    K = np.asarray(K, dtype=np.float64)
    ns = E.shape[0]
    return {
        "name": name,
        "n_states": ns,
        "n_modes": K.shape[0],
        "hbar": float(hbar),
        "mass": np.asarray(mass, dtype=np.float64),
        "omega": np.asarray(omega, dtype=np.float64),
        "E": np.asarray(E, dtype=np.float64),
        "K": K,
        "hop_scale": float(hop_scale),
        "p_max": float(p_max),
    }


def ohmic_modes(n_modes: int, xi: float, wc: float):
    j = np.arange(1, n_modes + 1, dtype=np.float64)
    omega = -wc * np.log(1.0 - j / (n_modes + 1))
    c = omega * math.sqrt(xi * wc / (n_modes + 1))
    return omega, c


def spin_boson(eps, delta, omega, c, mass=None, hbar=1.0, name="spin-boson", **kw):
    omega = np.asarray(omega, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    mass = np.ones_like(omega) if mass is None else np.asarray(mass, dtype=np.float64)
    E = eps * SZ + delta * SX
    K = c[:, None, None] * SZ[None, :, :]
    return _model(E, K, mass, omega, hbar=hbar, name=name, **kw)


def sb_init(model, beta=math.inf, state=0, wigner=1):
    """Diabatic |state><state|, bath equilibrated with that diabatic surface."""
    ns = model["n_states"]
    rho = np.zeros((ns, ns))
    rho[state, state] = 1.0
    k = model["mass"] * model["omega"] ** 2
    diag = model["K"][:, state, state]
    return {
        "rho_el0": rho,
        "R0": -diag / k,
        "P0": np.zeros(model["n_modes"]),
        "beta": float(beta),
        "wigner": int(wigner),
    }


def vibronic_ci(hop_scale=1.0, p_max=0.5):
    """Synthetic two-state three-mode LVC model with a conical intersection.
    Dimensionless normal coordinates mapped to R = q, P = hbar p,
    M_j = hbar^2 / w_j[eV], w_j = w_j[eV]/hbar (1/fs)."""
    w_ev = np.array([0.08, 0.12, 0.10])
    E = np.diag([-0.4, 0.4])
    k1 = np.array([-0.10, -0.20])
    k2 = np.array([0.15, 0.20])
    lam = 0.20
    K = np.zeros((3, 2, 2))
    K[0] = np.diag([k1[0], k2[0]])
    K[1] = np.diag([k1[1], k2[1]])
    K[2] = lam * SX
    mass = HBAR_EV_FS**2 / w_ev
    omega = w_ev / HBAR_EV_FS
    return _model(E, K, mass, omega, hbar=HBAR_EV_FS, hop_scale=hop_scale, p_max=p_max,
                  name="vibronic-ci-3mode")


def vibronic_init(model):
    return {
        "rho_el0": np.diag([0.0, 1.0]),
        "R0": np.zeros(3),
        "P0": np.zeros(3),
        "beta": math.inf,
        "wigner": 1,
    }


def random_lvc4(request_id: int, n_modes: int = 6):
    """Random four-state LVC model: unit masses, frequencies ~ U(0.5, 2),
    E = diag(0, 0.5, 1, 1.5), K_j with entries ~ U(0, 0.2) scaled by
    sqrt(6 / n_modes) (the six-mode coupling strength for any mode count)."""
    rng = np.random.default_rng(request_id)
    omega = rng.uniform(0.5, 2.0, size=n_modes)
    E = np.diag([0.0, 0.5, 1.0, 1.5])
    K = np.zeros((n_modes, 4, 4))
    scale = 1.0 if n_modes == 6 else math.sqrt(6.0 / n_modes)
    for j in range(n_modes):
        a = rng.uniform(0.0, 0.2, size=(4, 4)) * scale
        K[j] = np.triu(a) + np.triu(a, 1).T
    return _model(E, K, np.ones(n_modes), omega, name=f"random-lvc4-{request_id}")


def random_lvc2(n_modes: int, seed: int, scale: float = 0.3):
    """Random two-state LVC model with every gradient (s_j, a_j, b_j) nonzero:
    unit masses, frequencies ~ U(0.5, 2), E = [[0.3, 0.2], [0.2, -0.3]]."""
    rng = np.random.default_rng(seed)
    omega = rng.uniform(0.5, 2.0, size=n_modes)
    E = np.array([[0.3, 0.2], [0.2, -0.3]])
    K = np.zeros((n_modes, 2, 2))
    for j in range(n_modes):
        a, b, s = rng.normal(size=3) * scale / np.sqrt(n_modes) * omega[j]
        K[j] = np.array([[s + a, b], [b, s - a]])
    return _model(E, K, np.ones(n_modes), omega, name=f"random-lvc2-{n_modes}")


# --------------------------------------------------------------------- configs
def config(idx: int):
    """Returns dict(model, init, n_traj, dt, n_steps, out_stride, seed, precision)."""
    if idx == 1:
        m = spin_boson(0.0, 0.5, [1.0], [1.0], name="sb-1mode")
        return dict(name="sb1d", model=m, init=sb_init(m), n_traj=10_000, dt=0.01,
                    n_steps=1000, out_stride=10, seed=0, precision="fp64")
    if idx == 2:
        w, c = ohmic_modes(3, 0.5, 2.5)
        m = spin_boson(0.5, 0.5, w, c, name="sb-3mode-ohmic")
        return dict(name="sb3d", model=m, init=sb_init(m, beta=5.0), n_traj=10_000_000,
                    dt=0.01, n_steps=2000, out_stride=10, seed=0, precision="fp32")
    if idx == 3:
        m = vibronic_ci()
        return dict(name="vibronic3", model=m, init=vibronic_init(m), n_traj=100_000_000,
                    dt=0.05, n_steps=4000, out_stride=20, seed=0, precision="fp32")
    if idx == 4:
        w, c = ohmic_modes(100, 0.25, 5.0)
        m = spin_boson(1.0, 1.0, w, c, name="sb-100mode-ohmic")
        return dict(name="sb100", model=m, init=sb_init(m, beta=1.0), n_traj=10_000_000,
                    dt=0.005, n_steps=4000, out_stride=20, seed=0, precision="fp32")
    raise ValueError(idx)


def lvc4_config(request_id: int, n_modes: int = 6):
    m = random_lvc4(request_id, n_modes)
    return dict(name="lvc4", model=m, init=sb_init(m), n_traj=10_000, dt=0.01, n_steps=1000,
                out_stride=10, seed=request_id, precision="fp32")


def served_mix(n_requests: int = 256, mean_gap_s: float = 0.005, seed: int = 12345,
               traj_range=(1e4, 1e7), steps_range=(500, 4000)):
    """Poisson arrivals of requests drawn uniformly from the five model kinds."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(mean_gap_s, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(n_requests):
        kind = int(rng.integers(0, 5))
        if kind < 4:
            base = config(kind + 1)
        else:
            base = lvc4_config(i)
        lo, hi = math.log(traj_range[0]), math.log(traj_range[1])
        n_traj = int(round(math.exp(rng.uniform(lo, hi))))
        n_steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        stride = base["out_stride"]
        n_steps = max(stride, (n_steps // stride) * stride)
        reqs.append(dict(base, n_traj=n_traj, n_steps=n_steps, seed=i, precision="fp32",
                         arrival_s=float(t[i]), kind=kind, request_id=i))
    return reqs
