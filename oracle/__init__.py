"""FP64 CPU oracle for momentum-jump-free QCL dynamics (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or calls it, and
the oracle shares no code with it.

The oracle follows the paper's Eq. 1 (Sec. II A) one walker at a time; see
``qcl_oracle.c`` for the step-by-step statement of each reading.  Arrays cross
the boundary as contiguous numpy arrays, walker-major (``R[i, j]``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.environ.get("QCL_ORACLE_SRC", os.path.join(_HERE, "qcl_oracle.c"))
_LIB = os.environ.get("QCL_ORACLE_LIB", os.path.join(_HERE, "liboracle.so"))
_lib = None
_lock = threading.Lock()

PURPOSE_INIT = 1
PURPOSE_HOP = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "qcl_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
             "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Model(C.Structure):
    _fields_ = [
        ("n_states", C.c_int32), ("n_modes", C.c_int32), ("hbar", C.c_double),
        ("mass", C.c_void_p), ("omega", C.c_void_p), ("E", C.c_void_p), ("K", C.c_void_p),
        ("hop_scale", C.c_double), ("p_max", C.c_double), ("repr", C.c_int32),
        ("reserved", C.c_int32),
    ]


REPR_ADIABATIC = 0
REPR_DIABATIC = 1


def _repr_code(m: dict) -> int:
    r = m.get("repr", "adiabatic")
    if r in ("adiabatic", REPR_ADIABATIC):
        return REPR_ADIABATIC
    if r in ("diabatic", REPR_DIABATIC):
        return REPR_DIABATIC
    raise ValueError(f"unknown representation {r!r}")


class Init(C.Structure):
    _fields_ = [
        ("rho_el0", C.c_void_p), ("R0", C.c_void_p), ("P0", C.c_void_p),
        ("beta", C.c_double), ("wigner", C.c_int32),
    ]


def _l():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            vp, i32, i64, u64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
            lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
            lib.orc_jacobi_eigh.argtypes = [i32, vp, vp, vp]
            lib.orc_adiabatic.argtypes = [vp, vp, vp, vp, vp]
            lib.orc_adiabatic.restype = i32
            lib.orc_nac.argtypes = [vp, vp, vp, vp]
            lib.orc_mean_force.argtypes = [vp, vp, vp, i32, i32, vp]
            lib.orc_events.argtypes = [vp, vp, vp, vp, i32, i32, d, vp, vp, vp, vp]
            lib.orc_events.restype = i32
            lib.orc_events_dia.argtypes = [vp, vp, i32, i32, d, vp, vp, vp, vp, vp]
            lib.orc_events_dia.restype = i32
            lib.orc_step_deterministic.argtypes = [vp, vp, vp, vp, i32, i32, vp, d]
            lib.orc_sample.argtypes = [vp, vp, u64, u64, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_sample.restype = i32
            lib.orc_advance.argtypes = [vp, u64, u64, i64, vp, vp, vp, vp, vp, vp, vp, vp, i64,
                                        i64, d, vp]
            lib.orc_advance.restype = i32
            lib.orc_contrib.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_observe.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_run.argtypes = [vp, vp, u64, u64, i64, d, i64, i64, vp, vp]
            lib.orc_run.restype = i32
            lib.orc_spawn_sample.argtypes = [vp, vp, u64, u64, i64] + [vp] * 10
            lib.orc_spawn_sample.restype = i32
            lib.orc_spawn_advance.argtypes = [vp, u64, i64, vp] + [vp] * 10 + [i64, i64, d]
            lib.orc_spawn_advance.restype = i32
            lib.orc_spawn_observe.argtypes = [vp, i64, i64] + [vp] * 9
            lib.orc_run_spawn.argtypes = [vp, vp, u64, u64, i64, i64, d, i64, i64, vp, vp]
            lib.orc_run_spawn.restype = i32
            _lib = lib
    return _lib


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data if a is not None else None


class OracleModel:
    """Holds the model arrays alive for the C structure."""

    def __init__(self, m: dict):
        self.ns = int(m["n_states"])
        self.n = int(m["n_modes"])
        self.hbar = float(m["hbar"])
        self.mass = _f64(m["mass"])
        self.omega = _f64(m["omega"])
        self.E = _f64(m["E"]).reshape(self.ns * self.ns)
        self.K = _f64(m["K"]).reshape(self.n * self.ns * self.ns)
        self.hop_scale = float(m.get("hop_scale", 1.0))
        self.p_max = float(m.get("p_max", 0.5))
        self.repr = _repr_code(m)
        self.c = Model(self.ns, self.n, self.hbar, _ptr(self.mass), _ptr(self.omega),
                       _ptr(self.E), _ptr(self.K), self.hop_scale, self.p_max, self.repr, 0)

    @property
    def ref(self):
        return C.byref(self.c)


class OracleInit:
    def __init__(self, model: OracleModel, i: dict):
        self.rho = _f64(i["rho_el0"]).reshape(model.ns * model.ns)
        self.R0 = _f64(i["R0"]).reshape(model.n)
        self.P0 = _f64(i["P0"]).reshape(model.n)
        self.beta = float(i.get("beta", np.inf))
        self.wigner = int(i.get("wigner", 1))
        self.c = Init(_ptr(self.rho), _ptr(self.R0), _ptr(self.P0), self.beta, self.wigner)

    @property
    def ref(self):
        return C.byref(self.c)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _l().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def jacobi_eigh(A):
    A = _f64(A)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    _l().orc_jacobi_eigh(n, _ptr(A), _ptr(w), _ptr(V))
    return w, V


def adiabatic(model: OracleModel, R, U_ref=None):
    R = _f64(R)
    e = np.zeros(model.ns)
    U = np.zeros((model.ns, model.ns))
    Ur = _f64(U_ref) if U_ref is not None else None
    deg = _l().orc_adiabatic(model.ref, _ptr(R), _ptr(Ur), _ptr(e), _ptr(U))
    return e, U, deg


def nac(model: OracleModel, e, U):
    d = np.zeros((model.ns, model.ns, model.n))
    _l().orc_nac(model.ref, _ptr(_f64(e)), _ptr(_f64(U)), _ptr(d))
    return d


def mean_force(model: OracleModel, R, U, a, b):
    F = np.zeros(model.n)
    _l().orc_mean_force(model.ref, _ptr(_f64(R)), _ptr(_f64(U)), a, b, _ptr(F))
    return F


def events(model: OracleModel, P, e, U, a, b, dt):
    ne_max = 2 * model.ns
    ta = np.zeros(ne_max, dtype=np.int32)
    tb = np.zeros(ne_max, dtype=np.int32)
    A = np.zeros(ne_max)
    T = np.zeros(ne_max, dtype=np.uint32)
    ne = _l().orc_events(model.ref, _ptr(_f64(P)), _ptr(_f64(e)), _ptr(_f64(U)), a, b, dt,
                         _ptr(ta), _ptr(tb), _ptr(A), _ptr(T))
    return ta[:ne], tb[:ne], A[:ne], T[:ne]


def events_dia(model: OracleModel, R, a, b, dt):
    """Diabatic events: (target a, target b, real factor c, quarter turns, T)."""
    ne_max = 2 * model.ns
    ta = np.zeros(ne_max, dtype=np.int32)
    tb = np.zeros(ne_max, dtype=np.int32)
    c = np.zeros(ne_max)
    dq = np.zeros(ne_max, dtype=np.int32)
    T = np.zeros(ne_max, dtype=np.uint32)
    ne = _l().orc_events_dia(model.ref, _ptr(_f64(R)), a, b, dt, _ptr(ta), _ptr(tb), _ptr(c),
                             _ptr(dq), _ptr(T))
    return ta[:ne], tb[:ne], c[:ne], dq[:ne], T[:ne]


def step_deterministic(model: OracleModel, R, P, phi, a, b, U, dt):
    """Returns new (R, P, phi, U) after the deterministic part of one step."""
    R = _f64(R).copy()
    P = _f64(P).copy()
    ph = np.array([phi], dtype=np.float64)
    Uc = _f64(U).copy() if U is not None else None
    _l().orc_step_deterministic(model.ref, _ptr(R), _ptr(P), _ptr(ph), a, b, _ptr(Uc), dt)
    return R, P, float(ph[0]), Uc


class State:
    """Walker-major ensemble state of the oracle."""

    def __init__(self, model: OracleModel, n_traj: int):
        self.n_traj = n_traj
        self.R = np.zeros((n_traj, model.n))
        self.P = np.zeros((n_traj, model.n))
        self.m = np.zeros(n_traj)
        self.phi = np.zeros(n_traj)
        self.alpha = np.zeros(n_traj, dtype=np.int32)
        self.beta = np.zeros(n_traj, dtype=np.int32)
        self.U = np.zeros((n_traj, model.ns, model.ns))
        self.q = np.zeros(n_traj, dtype=np.int32)  # quarter turns (diabatic representation)

    def copy(self):
        s = State.__new__(State)
        for k, v in self.__dict__.items():
            setattr(s, k, v.copy() if isinstance(v, np.ndarray) else v)
        return s

    def args(self):
        return (_ptr(self.R), _ptr(self.P), _ptr(self.m), _ptr(self.phi), _ptr(self.alpha),
                _ptr(self.beta), _ptr(self.U), _ptr(self.q))


def sample(model: OracleModel, init: OracleInit, seed: int, traj_offset: int, n_traj: int):
    st = State(model, n_traj)
    rc = _l().orc_sample(model.ref, init.ref, seed, traj_offset, n_traj, *st.args())
    if rc != 0:
        raise ValueError("oracle: initial electronic density has no nonzero element")
    return st


def advance(model: OracleModel, st: State, seed: int, traj_offset: int, step0: int, n_steps: int,
            dt: float):
    ndeg = np.zeros(1, dtype=np.int64)
    _l().orc_advance(model.ref, seed, traj_offset, st.n_traj, *st.args(), step0, n_steps, dt,
                     _ptr(ndeg))
    return int(ndeg[0])


def contrib(model: OracleModel, st: State):
    q = np.zeros((st.n_traj, 4 * model.ns * model.ns))
    _l().orc_contrib(model.ref, st.n_traj, _ptr(st.R), _ptr(st.m), _ptr(st.phi),
                     _ptr(st.alpha), _ptr(st.beta), _ptr(st.U), _ptr(st.q), _ptr(q))
    return q


def observe(model: OracleModel, st: State):
    row = np.zeros(8 * model.ns * model.ns)
    _l().orc_observe(model.ref, st.n_traj, _ptr(st.R), _ptr(st.m), _ptr(st.phi),
                     _ptr(st.alpha), _ptr(st.beta), _ptr(st.U), _ptr(st.q), _ptr(row))
    return row


def run(model: OracleModel, init: OracleInit, seed: int, traj_offset: int, n_traj: int, dt: float,
        n_steps: int, out_stride: int):
    """Whole run; returns (rows[n_out, 8 NS^2] of sums and sums of squares, n_degenerate)."""
    n_out = n_steps // out_stride + 1
    rows = np.zeros((n_out, 8 * model.ns * model.ns))
    ndeg = np.zeros(1, dtype=np.int64)
    rc = _l().orc_run(model.ref, init.ref, seed, traj_offset, n_traj, dt, n_steps, out_stride,
                      _ptr(rows), _ptr(ndeg))
    if rc != 0:
        raise ValueError("oracle: initial electronic density has no nonzero element")
    return rows, int(ndeg[0])


def run_threaded(model: OracleModel, init: OracleInit, seed: int, n_traj: int, dt: float,
                 n_steps: int, out_stride: int, threads: int):
    """Static split of the walkers over host threads (ctypes releases the GIL).
    Returns the per-thread row sums added in thread order."""
    bounds = [n_traj * t // threads for t in range(threads + 1)]
    outs = [None] * threads

    def work(t):
        outs[t] = run(model, init, seed, bounds[t], bounds[t + 1] - bounds[t], dt, n_steps,
                      out_stride)[0]

    ths = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    total = outs[0].copy()
    for t in range(1, threads):
        total += outs[t]
    return total


def finalize(rows: np.ndarray, n_traj: int):
    """Means and standard errors from sums and sums of squares (divide by N)."""
    nq = rows.shape[1] // 2
    s, s2 = rows[:, :nq], rows[:, nq:]
    mean = s / n_traj
    var = np.maximum(s2 - s * s / n_traj, 0.0) / max(n_traj - 1, 1)
    se = np.sqrt(var / n_traj)
    return mean, se


# ------------------------------------------------------------------ spawning --
class SpawnState(State):
    """Spawning ensemble: arrays of `capacity` walkers, the first n_live live (in
    family order), with each walker's random-stream id and family index."""

    def __init__(self, model: OracleModel, n0: int, capacity: int):
        super().__init__(model, capacity)
        self.n0 = n0
        self.capacity = capacity
        self.n_live = n0
        self.id = np.zeros(capacity, dtype=np.uint64)
        self.family = np.zeros(capacity, dtype=np.int64)

    def sargs(self):
        return self.args() + (_ptr(self.id), _ptr(self.family))

    def live(self):
        """Dict of the live walkers' arrays."""
        k = self.n_live
        return {"R": self.R[:k], "P": self.P[:k], "m": self.m[:k], "phi": self.phi[:k],
                "alpha": self.alpha[:k], "beta": self.beta[:k], "q": self.q[:k],
                "id": self.id[:k], "family": self.family[:k]}


def spawn_sample(model: OracleModel, init: OracleInit, seed: int, traj_offset: int, n0: int,
                 capacity: int):
    st = SpawnState(model, n0, capacity)
    rc = _l().orc_spawn_sample(model.ref, init.ref, seed, traj_offset, n0, *st.sargs())
    if rc != 0:
        raise ValueError("oracle: initial electronic density has no nonzero element")
    return st


def spawn_advance(model: OracleModel, st: SpawnState, seed: int, step0: int, n_steps: int,
                  dt: float) -> int:
    """Returns 0, or -2 on capacity overflow."""
    nl = np.array([st.n_live], dtype=np.int64)
    rc = _l().orc_spawn_advance(model.ref, seed, st.capacity, _ptr(nl), *st.sargs(), step0,
                                n_steps, dt)
    st.n_live = int(nl[0])
    return rc


def spawn_observe(model: OracleModel, st: SpawnState):
    row = np.zeros(8 * model.ns * model.ns)
    _l().orc_spawn_observe(model.ref, st.n0, st.n_live, _ptr(st.R), _ptr(st.m), _ptr(st.phi),
                           _ptr(st.alpha), _ptr(st.beta), _ptr(st.U), _ptr(st.q),
                           _ptr(st.family), _ptr(row))
    return row


def run_spawn(model: OracleModel, init: OracleInit, seed: int, traj_offset: int, n0: int,
              capacity: int, dt: float, n_steps: int, out_stride: int):
    """Whole spawning run: (rows[n_out, 8 NS^2] of family sums and their squares,
    live walkers at each output).  Raises OverflowError past capacity."""
    n_out = n_steps // out_stride + 1
    rows = np.zeros((n_out, 8 * model.ns * model.ns))
    n_live = np.zeros(n_out, dtype=np.int64)
    rc = _l().orc_run_spawn(model.ref, init.ref, seed, traj_offset, n0, capacity, dt, n_steps,
                            out_stride, _ptr(rows), _ptr(n_live))
    if rc == -2:
        raise OverflowError("oracle: spawning ensemble exceeded its capacity")
    if rc != 0:
        raise ValueError("oracle: initial electronic density has no nonzero element")
    return rows, n_live
