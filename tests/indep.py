"""Independent numpy references used to pin the oracle.

None of these retype the oracle's formulas: eigenvectors come from
numpy.linalg.eigh, couplings and forces from finite differences of that
decomposition, and the harmonic propagator from powers of the 2x2 velocity
Verlet matrix.
"""
from __future__ import annotations

import numpy as np


def elec(model, R):
    return model["E"] + np.tensordot(R, model["K"], axes=(0, 0))


def eigh_aligned(model, R, ref=None):
    e, U = np.linalg.eigh(elec(model, R))
    if ref is not None:
        s = np.sign(np.sum(U * ref, axis=0))
        s[s == 0] = 1.0
        U = U * s
    return e, U


def nac_fd(model, R, h=1e-5):
    """d[mu, nu, j] = <mu | d nu / dR_j> by central differences of gauge-aligned
    eigenvectors."""
    n = model["n_modes"]
    ns = model["n_states"]
    e, U = eigh_aligned(model, R)
    d = np.zeros((ns, ns, n))
    for j in range(n):
        dR = np.zeros(n)
        dR[j] = h
        _, Up = eigh_aligned(model, R + dR, U)
        _, Um = eigh_aligned(model, R - dR, U)
        dU = (Up - Um) / (2 * h)
        d[:, :, j] = U.T @ dU
    return e, U, d


def mean_force_fd(model, R, a, b, h=1e-5):
    """-d/dR_j of 1/2 sum k R^2 + (e_a + e_b)/2 by central differences."""
    k = model["mass"] * model["omega"] ** 2
    n = model["n_modes"]
    F = np.zeros(n)
    for j in range(n):
        dR = np.zeros(n)
        dR[j] = h
        ep = np.linalg.eigvalsh(elec(model, R + dR))
        em = np.linalg.eigvalsh(elec(model, R - dR))
        F[j] = -k[j] * R[j] - 0.5 * ((ep[a] - em[a]) + (ep[b] - em[b])) / (2 * h)
    return F


def coupling_operator(model, P, d):
    """Matrix L of the coupling term of Eq. 1 acting on the vector of elements
    rho_(a,b) (row-major pair index): (L rho)_ab = -(P/M) sum_g (d_ag rho_gb -
    rho_ag d_gb)."""
    ns = model["n_states"]
    v = P / model["mass"]
    vd = np.tensordot(d, v, axes=(2, 0))  # vd[mu, nu] = sum_j v_j d_{mu nu, j}
    L = np.zeros((ns * ns, ns * ns))
    for a in range(ns):
        for b in range(ns):
            for g in range(ns):
                L[a * ns + b, g * ns + b] += -vd[a, g]
                L[a * ns + b, a * ns + g] += vd[g, b]
    return L


def verlet_matrix(omega, mass, dt):
    """Velocity Verlet map of (R, P) for a harmonic mode with force -k R."""
    k = mass * omega**2
    kick = np.array([[1.0, 0.0], [-0.5 * dt * k, 1.0]])
    drift = np.array([[1.0, dt / mass], [0.0, 1.0]])
    return kick @ drift @ kick
