"""The seeded synthetic workloads (stand-ins for the paper's model systems):
their construction against the stated recipe, without a GPU."""
import numpy as np
import pytest

from paper_2608_14544_gb300 import workloads as wl


@pytest.mark.parametrize("n,xi,wc", [(3, 0.5, 2.5), (100, 0.25, 5.0), (1, 1.0, 1.0)])
def test_ohmic_discretisation_reproduces_the_reorganisation_energy(n, xi, wc):
    # J(w) = (pi/2) xi w exp(-w/wc) with equal density of modes: the discrete
    # reorganisation energy sum_j c_j^2 / (2 w_j^2) is n/(n+1) of the
    # continuum's (1/pi) int J(w)/w dw = xi wc / 2, and the frequencies are
    # the (j/(n+1)) quantiles of the density exp(-w/wc)/wc
    w, c = wl.ohmic_modes(n, xi, wc)
    assert np.all(np.diff(w) > 0) and np.all(w > 0)
    assert np.sum(c**2 / (2 * w**2)) == pytest.approx(n / (n + 1) * xi * wc / 2, rel=1e-12)
    q = 1.0 - np.exp(-w / wc)
    assert np.allclose(q, np.arange(1, n + 1) / (n + 1), rtol=0, atol=1e-14)


def test_spin_boson_model_is_the_lvc_form():
    w, c = wl.ohmic_modes(3, 0.5, 2.5)
    m = wl.spin_boson(0.5, 0.25, w, c)
    assert m["n_states"] == 2 and m["n_modes"] == 3
    E, K = np.asarray(m["E"]), np.asarray(m["K"])
    assert np.allclose(E, [[0.5, 0.25], [0.25, -0.5]])  # eps sigma_z + Delta sigma_x
    for j in range(3):  # c_j sigma_z
        assert np.allclose(K[j], [[c[j], 0.0], [0.0, -c[j]]])


def test_random_lvc2_is_seeded_symmetric_and_fully_coupled():
    a, b = wl.random_lvc2(7, seed=3), wl.random_lvc2(7, seed=3)
    assert np.array_equal(np.asarray(a["K"]), np.asarray(b["K"]))
    assert not np.array_equal(np.asarray(a["K"]), np.asarray(wl.random_lvc2(7, seed=4)["K"]))
    K = np.asarray(a["K"])
    assert np.allclose(K, np.swapaxes(K, 1, 2))
    assert np.all(K[:, 0, 1] != 0) and np.all(K[:, 0, 0] != K[:, 1, 1])


@pytest.mark.parametrize("idx,n_states,n_modes,n_traj,dt,steps,stride",
                         [(1, 2, 1, 10_000, 0.01, 1000, 10), (2, 2, 3, 10_000_000, 0.01, 2000, 10),
                          (4, 2, 100, 10_000_000, 0.005, 4000, 20)])
def test_benchmark_workload_sizes(idx, n_states, n_modes, n_traj, dt, steps, stride):
    cfg = wl.config(idx)
    assert cfg["model"]["n_states"] == n_states and cfg["model"]["n_modes"] == n_modes
    assert (cfg["n_traj"], cfg["dt"], cfg["n_steps"], cfg["out_stride"]) == (n_traj, dt, steps,
                                                                               stride)
