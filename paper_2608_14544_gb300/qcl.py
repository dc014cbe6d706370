"""Python binding of libqcl.so: the C ABI of include/qcl.h, one function per
entry point with the same name.  Argument marshalling only: every step of the
propagation runs in the library's CUDA kernels.  Device buffers are torch
tensors (torch provides device memory and streams); host arrays are numpy.

The binding fails loudly if the library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqcl.so")

QCL_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OUT_OF_MEMORY", 4: "CUDA",
                5: "TIMEOUT", 6: "NUMERICAL", 7: "BUSY", 8: "NOT_FOUND"}
PREC_FP64 = 0
PREC_FP32_BULK = 1
OPT_GRID_CAP = 1
OPT_TIMING = 2
OPT_MODES_IN_MEMORY = 3
KERNEL_BULK, KERNEL_FP64_STEP = 0, 1
FLAG_NONFINITE, FLAG_DEGENERATE, FLAG_STEP_MISMATCH = 1, 2, 4

# every entry point declared in include/qcl.h (checked by the CPU test suite)
EXPORTS = [
    "qcl_last_error", "qcl_version", "qcl_set_option", "qcl_launch_count", "qcl_kernel_time",
    "qcl_create_model", "qcl_destroy_model", "qcl_ensemble_bytes", "qcl_obs_bytes",
    "qcl_ensemble_layout", "qcl_sample_initial", "qcl_propagate", "qcl_reduce_observables",
    "qcl_finalize_observables",
    "qcl_read_sums", "qcl_ensemble_status", "qcl_ensemble_restore", "qcl_propagate_noalloc",
    "qcl_server_create", "qcl_server_submit", "qcl_server_poll", "qcl_server_wait",
    "qcl_server_stats", "qcl_server_destroy", "qcl_shard_tile_walkers", "qcl_combine_shards",
    "qcl_spawn_bytes", "qcl_spawn_layout", "qcl_spawn_sample", "qcl_spawn_propagate",
    "qcl_spawn_live", "qcl_shard_chunk_walkers", "qcl_read_chunk_sums", "qcl_set_launch_shape", "qcl_get_launch_shape", "qcl_autotune_bytes",
    "qcl_autotune", "qcl_measure_peak",
]
FLAG_SPAWN_OVERFLOW = 8
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_ERROR = 0, 1, 2, 3


class QclError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ModelDesc(C.Structure):
    _fields_ = [("n_states", C.c_int32), ("n_modes", C.c_int32), ("hbar", C.c_double),
                ("mass", C.c_void_p), ("omega", C.c_void_p), ("E", C.c_void_p),
                ("K", C.c_void_p), ("hop_scale", C.c_double), ("p_max", C.c_double),
                ("repr", C.c_int32), ("reserved", C.c_int32)]


REPR_ADIABATIC = 0
REPR_DIABATIC = 1


def repr_code(m: dict) -> int:
    """QCL_REPR_* of a model dict ("repr": "adiabatic" (default) or "diabatic")."""
    r = m.get("repr", "adiabatic")
    if r in ("adiabatic", REPR_ADIABATIC):
        return REPR_ADIABATIC
    if r in ("diabatic", REPR_DIABATIC):
        return REPR_DIABATIC
    raise ValueError(f"unknown representation {r!r}")


class LaunchShape(C.Structure):
    _fields_ = [("walkers_per_thread", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("walker_steps_per_s", C.c_double), ("outputs_per_launch", C.c_int32),
                ("reserved", C.c_int32)]


class EnsembleDesc(C.Structure):
    _fields_ = [("n_traj", C.c_int64), ("seed", C.c_uint64), ("traj_id_offset", C.c_uint64),
                ("precision", C.c_int32), ("reserved", C.c_int32)]


class InitDesc(C.Structure):
    _fields_ = [("rho_el0", C.c_void_p), ("R0", C.c_void_p), ("P0", C.c_void_p),
                ("beta", C.c_double), ("wigner", C.c_int32), ("reserved", C.c_int32)]


class ServerDesc(C.Structure):
    _fields_ = [("arena", C.c_void_p), ("arena_bytes", C.c_size_t), ("max_active", C.c_int32),
                ("quantum_steps", C.c_int32), ("use_graphs", C.c_int32), ("max_queue", C.c_int32),
                ("round_timeout_s", C.c_double), ("round_flops", C.c_double)]


class RequestDesc(C.Structure):
    _fields_ = [("model", C.c_void_p), ("init", C.c_void_p), ("n_traj", C.c_int64),
                ("seed", C.c_uint64), ("traj_id_offset", C.c_uint64), ("n_steps", C.c_int64),
                ("dt", C.c_double), ("out_stride", C.c_int32), ("reserved", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("n_submitted", C.c_int64), ("n_done", C.c_int64), ("n_error", C.c_int64),
                ("n_active", C.c_int64), ("n_queued", C.c_int64), ("rounds", C.c_int64),
                ("graph_replays", C.c_int64), ("arena_used", C.c_size_t),
                ("traj_steps_done", C.c_double), ("latency_p50_s", C.c_double),
                ("latency_p99_s", C.c_double), ("latency_mean_s", C.c_double),
                ("span_s", C.c_double), ("throughput", C.c_double),
                ("device_busy_s", C.c_double), ("device_throughput", C.c_double)]


class EnsStatus(C.Structure):
    _fields_ = [("step", C.c_int64), ("flags", C.c_uint32), ("reserved", C.c_uint32),
                ("n_degenerate", C.c_uint64), ("n_nonfinite", C.c_uint64)]


_lib = None


def load(path: str = LIB_PATH):
    """Loads libqcl.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libqcl.so not built at {path}: run __graft_entry__.build() "
                          "(the CUDA library is required; there is no CPU fallback)")
    lib = C.CDLL(path)
    vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
    lib.qcl_last_error.restype = C.c_char_p
    lib.qcl_version.restype = C.c_char_p
    lib.qcl_set_option.argtypes = [i32, i64]
    lib.qcl_launch_count.argtypes = [vp, i32]
    lib.qcl_kernel_time.argtypes = [i32, vp, vp]
    lib.qcl_ensemble_layout.argtypes = [vp, vp, vp]
    lib.qcl_create_model.argtypes = [vp, vp]
    lib.qcl_destroy_model.argtypes = [vp]
    lib.qcl_ensemble_bytes.argtypes = [vp, vp, vp]
    lib.qcl_obs_bytes.argtypes = [vp, vp, i64, vp]
    lib.qcl_sample_initial.argtypes = [vp, vp, vp, vp, sz, vp]
    lib.qcl_propagate.argtypes = [vp, vp, vp, sz, i64, i64, C.c_double, i32, vp, sz, i64, vp]
    lib.qcl_reduce_observables.argtypes = [vp, vp, vp, sz, i64, i64, i64, vp, sz, vp]
    lib.qcl_finalize_observables.argtypes = [vp, vp, vp, sz, i64, i64, i64, vp, sz, vp]
    lib.qcl_read_sums.argtypes = [vp, vp, vp, sz, i64, i64, i64, vp, sz, vp]
    lib.qcl_ensemble_status.argtypes = [vp, vp, vp, sz, vp, vp]
    lib.qcl_ensemble_restore.argtypes = [vp, vp, vp, sz, i64, vp]
    lib.qcl_propagate_noalloc.argtypes = [vp, vp, vp, sz, i64, i64, C.c_double, i32, vp, sz, i64,
                                          vp]
    lib.qcl_shard_tile_walkers.argtypes = [vp, i32, vp]
    lib.qcl_combine_shards.argtypes = [vp, i32, i64, vp]
    lib.qcl_shard_chunk_walkers.argtypes = [vp, i32, vp]
    lib.qcl_read_chunk_sums.argtypes = [vp, vp, vp, sz, i64, i64, i64, vp, sz, vp, vp]
    lib.qcl_server_create.argtypes = [vp, vp]
    lib.qcl_server_submit.argtypes = [vp, vp, vp]
    lib.qcl_server_poll.argtypes = [vp, i64, vp, vp, sz, vp]
    lib.qcl_server_wait.argtypes = [vp, i64, C.c_double, vp]
    lib.qcl_server_stats.argtypes = [vp, vp]
    lib.qcl_server_destroy.argtypes = [vp]
    lib.qcl_spawn_bytes.argtypes = [vp, vp, i64, vp]
    lib.qcl_spawn_layout.argtypes = [vp, vp, i64, i32, vp]
    lib.qcl_spawn_sample.argtypes = [vp, vp, vp, i64, vp, sz, vp]
    lib.qcl_spawn_propagate.argtypes = [vp, vp, i64, vp, sz, i64, i64, C.c_double, i32, vp, sz,
                                        i64, vp]
    lib.qcl_spawn_live.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.qcl_set_launch_shape.argtypes = [vp, vp]
    lib.qcl_get_launch_shape.argtypes = [vp, vp]
    lib.qcl_autotune_bytes.argtypes = [vp, i64, i64, i32, vp]
    lib.qcl_autotune.argtypes = [vp, i64, i64, C.c_double, i32, vp, sz, vp, vp]
    lib.qcl_measure_peak.argtypes = [i32, vp, vp]
    for name in EXPORTS:
        f = getattr(lib, name)
        if name not in ("qcl_last_error", "qcl_version"):
            f.restype = i32
    _lib = lib
    return lib


def _check(st: int, fn: str):
    if st != QCL_OK:
        raise QclError(st, fn, load().qcl_last_error().decode())


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _stream_ptr(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _dptr(t) -> int:
    return t.data_ptr() if hasattr(t, "data_ptr") else int(t)


def last_error() -> str:
    return load().qcl_last_error().decode()


def version() -> str:
    return load().qcl_version().decode()


def set_option(key: int, value: int):
    """Process-wide option (include/qcl.h): OPT_GRID_CAP (cap on the persistent
    grid, 0 = none), OPT_TIMING (1: CUDA events around the kernel launches),
    OPT_MODES_IN_MEMORY (0: the measured choice between the register and
    modes-in-memory kernels, 1: memory, 2: registers where a form exists).  No
    option changes a bit of any result."""
    _check(load().qcl_set_option(key, value), "qcl_set_option")


def launch_count(reset: bool = False) -> int:
    c = C.c_int64()
    _check(load().qcl_launch_count(C.byref(c), 1 if reset else 0), "qcl_launch_count")
    return c.value


def kernel_time(which: int):
    """(total ms, launches) recorded under OPT_TIMING for a kernel class."""
    ms, n = C.c_double(), C.c_int64()
    _check(load().qcl_kernel_time(which, C.byref(ms), C.byref(n)), "qcl_kernel_time")
    return ms.value, n.value


def ensemble_layout(model, ens) -> list:
    off = (C.c_size_t * 11)()
    _check(load().qcl_ensemble_layout(model.handle, C.byref(ens), off), "qcl_ensemble_layout")
    return list(off)


class Model:
    """Owns a qcl_model handle (create_model / destroy_model)."""

    def __init__(self, m: dict):
        self.ns = int(m["n_states"])
        self.n = int(m["n_modes"])
        self._arrs = [_f64(m["mass"]), _f64(m["omega"]), _f64(m["E"]).reshape(-1),
                      _f64(m["K"]).reshape(-1)]
        d = ModelDesc(self.ns, self.n, float(m["hbar"]), *[a.ctypes.data for a in self._arrs],
                      float(m.get("hop_scale", 1.0)), float(m.get("p_max", 0.5)), repr_code(m), 0)
        h = C.c_void_p()
        _check(load().qcl_create_model(C.byref(d), C.byref(h)), "qcl_create_model")
        self.handle = h

    def close(self):
        if self.handle:
            load().qcl_destroy_model(self.handle)
            self.handle = None

    def set_launch_shape(self, walkers_per_thread: int = 0, blocks_per_sm: int = 0,
                         outputs_per_launch: int = 0):
        """Launch shape of the FP32-bulk kernels (0 = default); results do not
        depend on it."""
        sh = LaunchShape(int(walkers_per_thread), int(blocks_per_sm), 0.0,
                         int(outputs_per_launch), 0)
        _check(load().qcl_set_launch_shape(self.handle, C.byref(sh)), "qcl_set_launch_shape")

    @staticmethod
    def _shape_dict(sh) -> dict:
        return {"walkers_per_thread": sh.walkers_per_thread, "blocks_per_sm": sh.blocks_per_sm,
                "outputs_per_launch": sh.outputs_per_launch,
                "walker_steps_per_s": sh.walker_steps_per_s}

    def launch_shape(self) -> dict:
        sh = LaunchShape()
        _check(load().qcl_get_launch_shape(self.handle, C.byref(sh)), "qcl_get_launch_shape")
        return self._shape_dict(sh)

    def autotune(self, dt: float, out_stride: int, probe_walkers: int = 1 << 20,
                 n_steps: int = 160, stream=None) -> dict:
        """Times the candidate launch shapes on a probe ensemble and keeps the
        fastest (see qcl_autotune); returns it with its measured rate."""
        b = C.c_size_t()
        _check(load().qcl_autotune_bytes(self.handle, probe_walkers, n_steps, out_stride,
                                         C.byref(b)), "qcl_autotune_bytes")
        scratch = device_buffer(b.value)
        sh = LaunchShape()
        _check(load().qcl_autotune(self.handle, probe_walkers, n_steps, dt, out_stride,
                                   _dptr(scratch), b.value, C.byref(sh), _stream_ptr(stream)),
               "qcl_autotune")
        del scratch
        return self._shape_dict(sh)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_model(m: dict) -> Model:
    return Model(m)


def destroy_model(model: Model):
    model.close()


def ens_desc(n_traj: int, seed: int, precision: int, traj_id_offset: int = 0) -> EnsembleDesc:
    return EnsembleDesc(int(n_traj), int(seed), int(traj_id_offset), int(precision), 0)


def ensemble_bytes(model: Model, ens: EnsembleDesc) -> int:
    b = C.c_size_t()
    _check(load().qcl_ensemble_bytes(model.handle, C.byref(ens), C.byref(b)),
           "qcl_ensemble_bytes")
    return b.value


def obs_bytes(model: Model, ens: EnsembleDesc, n_out: int) -> int:
    b = C.c_size_t()
    _check(load().qcl_obs_bytes(model.handle, C.byref(ens), n_out, C.byref(b)), "qcl_obs_bytes")
    return b.value


def sample_initial(model: Model, ens: EnsembleDesc, init: dict, ens_buf, stream=None):
    arrs = [_f64(init["rho_el0"]).reshape(-1), _f64(init["R0"]), _f64(init["P0"])]
    d = InitDesc(*[a.ctypes.data for a in arrs], float(init.get("beta", math.inf)),
                 int(init.get("wigner", 1)), 0)
    _check(load().qcl_sample_initial(model.handle, C.byref(ens), C.byref(d), _dptr(ens_buf),
                                     ens_buf.numel() * ens_buf.element_size(),
                                     _stream_ptr(stream)), "qcl_sample_initial")


def propagate(model: Model, ens: EnsembleDesc, ens_buf, step0: int, n_steps: int, dt: float,
              out_stride: int, obs_buf, n_out: int, stream=None):
    _check(load().qcl_propagate(model.handle, C.byref(ens), _dptr(ens_buf),
                                ens_buf.numel() * ens_buf.element_size(), step0, n_steps, dt,
                                out_stride, _dptr(obs_buf), obs_buf.numel() * obs_buf.element_size(),
                                n_out, _stream_ptr(stream)), "qcl_propagate")


def propagate_noalloc(model: Model, ens: EnsembleDesc, ens_buf, step0: int, n_steps: int,
                      dt: float, out_stride: int, rows, n_out: int, stream=None):
    """qcl_propagate_noalloc: FP32-bulk propagation whose scratch lives in the
    library's static device array; `rows` is a caller-owned device tensor of
    n_out x 8 NS^2 float64 that receives the output rows."""
    _check(load().qcl_propagate_noalloc(model.handle, C.byref(ens), _dptr(ens_buf),
                                        ens_buf.numel() * ens_buf.element_size(), step0, n_steps,
                                        dt, out_stride, _dptr(rows),
                                        rows.numel() * rows.element_size(), n_out,
                                        _stream_ptr(stream)), "qcl_propagate_noalloc")


def reduce_observables(model: Model, ens: EnsembleDesc, obs_buf, n_out: int, k0: int = 0,
                       n_rows: int | None = None, stream=None) -> np.ndarray:
    n_rows = n_out - k0 if n_rows is None else n_rows
    q = 4 * model.ns * model.ns
    out = np.zeros((n_rows, 2 * q + 3))
    _check(load().qcl_reduce_observables(model.handle, C.byref(ens), _dptr(obs_buf),
                                         obs_buf.numel() * obs_buf.element_size(), n_out, k0,
                                         n_rows, out.ctypes.data, out.size,
                                         _stream_ptr(stream)), "qcl_reduce_observables")
    return out


def finalize_observables(model: Model, ens: EnsembleDesc, obs_buf, n_out: int, dev_out,
                         k0: int = 0, n_rows: int | None = None, stream=None):
    """Means and standard errors into the device tensor dev_out (float64,
    [n_rows, 2Q + 3]), enqueued on `stream` without synchronising."""
    n_rows = n_out - k0 if n_rows is None else n_rows
    _check(load().qcl_finalize_observables(model.handle, C.byref(ens), _dptr(obs_buf),
                                           obs_buf.numel() * obs_buf.element_size(), n_out, k0,
                                           n_rows, _dptr(dev_out), dev_out.numel(),
                                           _stream_ptr(stream)), "qcl_finalize_observables")
    return dev_out


def read_sums(model: Model, ens: EnsembleDesc, obs_buf, n_out: int, k0: int = 0,
              n_rows: int | None = None, stream=None) -> np.ndarray:
    n_rows = n_out - k0 if n_rows is None else n_rows
    out = np.zeros((n_rows, 8 * model.ns * model.ns))
    _check(load().qcl_read_sums(model.handle, C.byref(ens), _dptr(obs_buf),
                                obs_buf.numel() * obs_buf.element_size(), n_out, k0, n_rows,
                                out.ctypes.data, out.size, _stream_ptr(stream)), "qcl_read_sums")
    return out


def ensemble_status(model: Model, ens: EnsembleDesc, ens_buf, stream=None) -> dict:
    s = EnsStatus()
    _check(load().qcl_ensemble_status(model.handle, C.byref(ens), _dptr(ens_buf),
                                      ens_buf.numel() * ens_buf.element_size(), C.byref(s),
                                      _stream_ptr(stream)), "qcl_ensemble_status")
    return {"step": s.step, "flags": s.flags, "n_degenerate": s.n_degenerate,
            "n_nonfinite": s.n_nonfinite}


def ensemble_restore(model: Model, ens: EnsembleDesc, ens_buf, step: int, stream=None):
    """qcl_ensemble_restore: the header of an ensemble at absolute step `step`
    whose walker arrays the caller has written."""
    _check(load().qcl_ensemble_restore(model.handle, C.byref(ens), _dptr(ens_buf),
                                       ens_buf.numel() * ens_buf.element_size(), int(step),
                                       _stream_ptr(stream)), "qcl_ensemble_restore")


# ------------------------------------------------------------- conveniences --
def device_buffer(nbytes: int, device="cuda"):
    """Caller-owned device memory from torch (256-byte aligned)."""
    import torch

    t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)
    if t.data_ptr() % 256:
        raise RuntimeError("torch returned a buffer that is not 256-byte aligned")
    return t


class Run:
    """One ensemble with its device buffers: sample, propagate, observe."""

    def __init__(self, model: Model, n_traj: int, seed: int, precision: int, n_out: int,
                 traj_id_offset: int = 0, device="cuda"):
        self.model = model
        self.ens = ens_desc(n_traj, seed, precision, traj_id_offset)
        self.n_out = n_out
        self.ens_buf = device_buffer(ensemble_bytes(model, self.ens), device)
        self.obs_buf = device_buffer(obs_bytes(model, self.ens, n_out), device)
        self.step = 0

    def sample(self, init: dict, stream=None):
        sample_initial(self.model, self.ens, init, self.ens_buf, stream)
        self.step = 0

    def propagate(self, n_steps: int, dt: float, out_stride: int, stream=None):
        propagate(self.model, self.ens, self.ens_buf, self.step, n_steps, dt, out_stride,
                  self.obs_buf, self.n_out, stream)
        self.step += n_steps

    def observables(self, stream=None) -> np.ndarray:
        return reduce_observables(self.model, self.ens, self.obs_buf, self.n_out, stream=stream)

    def observables_device(self, dev_out, stream=None):
        """observables() into a device float64 tensor, without a host copy."""
        return finalize_observables(self.model, self.ens, self.obs_buf, self.n_out, dev_out,
                                    stream=stream)

    def sums(self, stream=None) -> np.ndarray:
        return read_sums(self.model, self.ens, self.obs_buf, self.n_out, stream=stream)

    def chunk_sums(self, stream=None) -> np.ndarray:
        return read_chunk_sums(self.model, self.ens, self.obs_buf, self.n_out, stream=stream)

    def status(self, stream=None) -> dict:
        return ensemble_status(self.model, self.ens, self.ens_buf, stream)

    def load_state(self, st: dict, step: int, stream=None):
        """Checkpoint restore: writes walker arrays already in this ensemble's
        precision and layout -- the dict state() returns: R, P [n_traj, n];
        m, m_lo, m_exp, phi, phi_lo, alpha, q, beta [n_traj]; U [n_traj, NS, NS]
        and E [n_traj, NS] for models of more than two states -- into the
        buffer, then qcl_ensemble_restore sets its step."""
        import torch

        nt, n, ns = self.ens.n_traj, self.model.n, self.model.ns
        off = ensemble_layout(self.model, self.ens)
        fp64 = self.ens.precision == PREC_FP64
        ft = np.float64 if fp64 else np.float32
        host = np.zeros(self.ens_buf.numel(), dtype=np.uint8)

        def put(o, a, dtype):
            b = np.ascontiguousarray(np.asarray(a, dtype=dtype)).view(np.uint8).reshape(-1)
            host[o:o + b.size] = b

        put(off[0], np.asarray(st["R"]).reshape(nt, n).T, ft)
        put(off[1], np.asarray(st["P"]).reshape(nt, n).T, ft)
        put(off[2], st["m"], ft)
        put(off[4], st["phi"], ft)
        if not fp64:
            put(off[3], st["m_lo"], ft)
            put(off[5], st["phi_lo"], ft)
            put(off[8], st["m_exp"], np.int32)
        ab = (np.asarray(st["alpha"]) | (np.asarray(st.get("q", 0)) << 4)
              | (np.asarray(st["beta"]) << 8))
        put(off[6], ab, np.uint16)
        if ns > 2:
            put(off[9], np.asarray(st["U"]).reshape(nt, ns * ns).T, ft)
            if not fp64:
                put(off[10], np.asarray(st["E"]).reshape(nt, ns).T, ft)
        self.ens_buf.copy_(torch.from_numpy(host).to(self.ens_buf.device))
        ensemble_restore(self.model, self.ens, self.ens_buf, step, stream)
        self.step = int(step)

    def state(self):
        """Host copy of the SoA walker state (for checkpoints and parity tests)."""
        import torch

        torch.cuda.synchronize()
        nt, n = self.ens.n_traj, self.model.n
        off = ensemble_layout(self.model, self.ens)
        raw = self.ens_buf.cpu().numpy()
        fp64 = self.ens.precision == PREC_FP64
        dt = np.float64 if fp64 else np.float32
        w = 8 if fp64 else 4

        def arr(o, count, dtype, width):
            return np.frombuffer(raw[o:o + width * count].tobytes(), dtype=dtype).copy()

        mexp = np.zeros(nt, dtype=np.int32) if fp64 else arr(off[8], nt, np.int32, 4)
        ns = self.model.ns
        extra = {}
        if ns > 2:
            extra["U"] = arr(off[9], nt * ns * ns, dt, w).reshape(ns, ns, nt).transpose(2, 0, 1).copy()
            if not fp64:
                extra["E"] = arr(off[10], nt * ns, dt, w).reshape(ns, nt).T.copy()
        return {"R": arr(off[0], nt * n, dt, w).reshape(n, nt).T.copy(), "m_exp": mexp,
                "P": arr(off[1], nt * n, dt, w).reshape(n, nt).T.copy(),
                "m": arr(off[2], nt, dt, w),
                "m_lo": np.zeros(nt) if fp64 else arr(off[3], nt, dt, w),
                "phi": arr(off[4], nt, dt, w),
                "phi_lo": np.zeros(nt) if fp64 else arr(off[5], nt, dt, w),
                # index pair word: alpha | q << 4 | beta << 8 (q: quarter turns of a
                # diabatic walker's weight, 0 in the adiabatic representation)
                "alpha": (arr(off[6], nt, np.uint16, 2) & 0xF).astype(np.int32),
                "q": ((arr(off[6], nt, np.uint16, 2) >> 4) & 0x3).astype(np.int32),
                "beta": (arr(off[6], nt, np.uint16, 2) >> 8).astype(np.int32), **extra}


def measure_peak(which: int, stream=None) -> float:
    """Measured FMA throughput of the device in flops/s: 0 = FP32, 1 = FP64."""
    v = C.c_double()
    _check(load().qcl_measure_peak(int(which), C.byref(v), _stream_ptr(stream)),
           "qcl_measure_peak")
    return v.value


# ----------------------------------------------------------------- spawning --
class SpawnRun:
    """A trajectory-spawning ensemble (FP64 for any number of states, or FP32
    bulk for two states with at most 32 modes and more states with at most 8):
    n0 initial walkers (families) in a buffer of `capacity` walker slots."""

    def __init__(self, model: Model, n0: int, capacity: int, seed: int, n_out: int,
                 traj_id_offset: int = 0, device="cuda", precision: int = None):
        self.model = model
        self.capacity = int(capacity)
        prec = PREC_FP64 if precision is None else int(precision)
        self.ens = ens_desc(n0, seed, prec, traj_id_offset)
        self.n_out = n_out
        b = C.c_size_t()
        _check(load().qcl_spawn_bytes(model.handle, C.byref(self.ens), self.capacity, C.byref(b)),
               "qcl_spawn_bytes")
        self.buf = device_buffer(b.value, device)
        self.obs_buf = device_buffer(obs_bytes(model, self.ens, n_out), device)
        self.step = 0

    def sample(self, init: dict, stream=None):
        d, keep = _init_desc(init)
        _check(load().qcl_spawn_sample(self.model.handle, C.byref(self.ens), C.byref(d),
                                       self.capacity, _dptr(self.buf), self.buf.numel(),
                                       _stream_ptr(stream)), "qcl_spawn_sample")
        self.step = 0

    def propagate(self, n_steps: int, dt: float, out_stride: int, stream=None):
        _check(load().qcl_spawn_propagate(self.model.handle, C.byref(self.ens), self.capacity,
                                          _dptr(self.buf), self.buf.numel(), self.step,
                                          n_steps, dt, out_stride, _dptr(self.obs_buf),
                                          self.obs_buf.numel(), self.n_out,
                                          _stream_ptr(stream)), "qcl_spawn_propagate")
        self.step += n_steps

    def n_live(self, stream=None) -> int:
        v = C.c_int64()
        _check(load().qcl_spawn_live(self.model.handle, C.byref(self.ens), self.capacity,
                                     _dptr(self.buf), C.byref(v), _stream_ptr(stream)),
               "qcl_spawn_live")
        return v.value

    def observables(self, stream=None) -> np.ndarray:
        return reduce_observables(self.model, self.ens, self.obs_buf, self.n_out, stream=stream)

    def sums(self, stream=None) -> np.ndarray:
        return read_sums(self.model, self.ens, self.obs_buf, self.n_out, stream=stream)

    def status(self, stream=None) -> dict:
        return ensemble_status(self.model, self.ens, self.buf, stream)

    def state(self) -> dict:
        """Host copy of the live walkers of the current set, in walker order."""
        import torch

        torch.cuda.synchronize()
        nl, n, cap = self.n_live(), self.model.n, self.capacity
        off = (C.c_size_t * 12)()
        _check(load().qcl_spawn_layout(self.model.handle, C.byref(self.ens), cap, self.step & 1,
                                       off), "qcl_spawn_layout")
        raw = self.buf.cpu().numpy()
        fp64 = self.ens.precision == PREC_FP64
        dt, w = (np.float64, 8) if fp64 else (np.float32, 4)

        def arr(o, count, dtype, width):
            return np.frombuffer(raw[o:o + width * count].tobytes(), dtype=dtype).copy()

        R = arr(off[0], n * cap, dt, w).reshape(n, cap)[:, :nl].T.copy()
        P = arr(off[1], n * cap, dt, w).reshape(n, cap)[:, :nl].T.copy()
        ab = arr(off[4], nl, np.uint16, 2)
        out = {"R": R, "P": P, "m": arr(off[2], nl, dt, w), "phi": arr(off[3], nl, dt, w),
               "alpha": (ab & 0xF).astype(np.int32), "q": ((ab >> 4) & 0x3).astype(np.int32),
               "beta": (ab >> 8).astype(np.int32), "id": arr(off[5], nl, np.uint64, 8),
               "family": arr(off[6], nl, np.uint32, 4).astype(np.int64)}
        if not fp64:
            out["m_lo"] = arr(off[8], nl, np.float32, 4)
            out["m_exp"] = arr(off[9], nl, np.int32, 4)
            out["phi_lo"] = arr(off[10], nl, np.float32, 4)
        ns = self.model.ns
        if ns > 2:
            out["U"] = arr(off[11], ns * ns * cap, dt, w).reshape(ns, ns, cap)[:, :, :nl]
            out["U"] = out["U"].transpose(2, 0, 1).copy()
        return out


# ------------------------------------------------------------------- shards --
def shard_tile_walkers(model: Model, precision: int) -> int:
    w = C.c_int64()
    _check(load().qcl_shard_tile_walkers(model.handle, precision, C.byref(w)),
           "qcl_shard_tile_walkers")
    return w.value


def shard_chunk_walkers(model: Model, precision: int) -> int:
    w = C.c_int64()
    _check(load().qcl_shard_chunk_walkers(model.handle, precision, C.byref(w)),
           "qcl_shard_chunk_walkers")
    return w.value


def read_chunk_sums(model: Model, ens: EnsembleDesc, obs_buf, n_out: int, k0: int = 0,
                    n_rows: int | None = None, stream=None) -> np.ndarray:
    """Per-chunk sums of output rows [k0, k0 + n_rows): [n_rows, chunks, 8 NS^2]."""
    n_rows = n_out - k0 if n_rows is None else n_rows
    nb = obs_buf.numel() * obs_buf.element_size()
    nc = C.c_int64()
    _check(load().qcl_read_chunk_sums(model.handle, C.byref(ens), _dptr(obs_buf), nb, n_out, k0,
                                      n_rows, None, 0, C.byref(nc), _stream_ptr(stream)),
           "qcl_read_chunk_sums")
    out = np.zeros((n_rows, nc.value, 8 * model.ns * model.ns))
    _check(load().qcl_read_chunk_sums(model.handle, C.byref(ens), _dptr(obs_buf), nb, n_out, k0,
                                      n_rows, out.ctypes.data, out.size, C.byref(nc),
                                      _stream_ptr(stream)), "qcl_read_chunk_sums")
    return out


def combine_shards(shard_sums) -> np.ndarray:
    """Binary-tree combine of per-shard output sums (first axis = shard, in
    walker order), the same tree as one unsharded run."""
    a = np.ascontiguousarray(np.asarray(shard_sums, dtype=np.float64))
    out = np.zeros(a.shape[1:])
    _check(load().qcl_combine_shards(a.ctypes.data, a.shape[0], int(out.size), out.ctypes.data),
           "qcl_combine_shards")
    return out


# ------------------------------------------------------------------ serving --
def _model_desc(m: dict):
    arrs = [_f64(m["mass"]), _f64(m["omega"]), _f64(m["E"]).reshape(-1), _f64(m["K"]).reshape(-1)]
    d = ModelDesc(int(m["n_states"]), int(m["n_modes"]), float(m["hbar"]),
                  *[a.ctypes.data for a in arrs], float(m.get("hop_scale", 1.0)),
                  float(m.get("p_max", 0.5)), repr_code(m), 0)
    return d, arrs


def _init_desc(i: dict):
    arrs = [_f64(i["rho_el0"]).reshape(-1), _f64(i["R0"]), _f64(i["P0"])]
    d = InitDesc(*[a.ctypes.data for a in arrs], float(i.get("beta", math.inf)),
                 int(i.get("wigner", 1)), 0)
    return d, arrs


class Server:
    """qcl_server_*: continuous-batching request loop over a caller-owned
    device arena (a torch tensor held by this object)."""

    def __init__(self, arena_bytes: int, max_active: int = 64, quantum_steps: int = 200,
                 use_graphs: bool = True, max_queue: int = 0, round_timeout_s: float = 0.0,
                 round_flops: float = 0.0, device="cuda"):
        self.arena = device_buffer(arena_bytes, device)
        d = ServerDesc(self.arena.data_ptr(), int(arena_bytes), int(max_active),
                       int(quantum_steps), 1 if use_graphs else 0, int(max_queue),
                       float(round_timeout_s), float(round_flops))
        h = C.c_void_p()
        _check(load().qcl_server_create(C.byref(d), C.byref(h)), "qcl_server_create")
        self.handle = h
        self.n_states = {}

    def submit(self, req: dict) -> int:
        md, keep1 = _model_desc(req["model"])
        ind, keep2 = _init_desc(req["init"])
        r = RequestDesc(C.addressof(md), C.addressof(ind), int(req["n_traj"]), int(req["seed"]),
                        int(req.get("traj_id_offset", 0)), int(req["n_steps"]), float(req["dt"]),
                        int(req["out_stride"]), 0)
        rid = C.c_int64()
        _check(load().qcl_server_submit(self.handle, C.byref(r), C.byref(rid)), "qcl_server_submit")
        self.n_states[rid.value] = int(req["model"]["n_states"])
        return rid.value

    def poll(self, rid: int):
        """(state, observables or None)."""
        st, n_rows = C.c_int32(), C.c_int64()
        _check(load().qcl_server_poll(self.handle, rid, C.byref(st), None, 0, C.byref(n_rows)),
               "qcl_server_poll")
        if st.value != REQ_DONE:
            return st.value, None
        q = 4 * self.n_states[rid] ** 2
        out = np.zeros((n_rows.value, 2 * q + 3))
        _check(load().qcl_server_poll(self.handle, rid, C.byref(st), out.ctypes.data, out.size,
                                      C.byref(n_rows)), "qcl_server_poll")
        return st.value, out

    def wait(self, rid: int, timeout_s: float = 600.0):
        st = C.c_int32()
        _check(load().qcl_server_wait(self.handle, rid, timeout_s, C.byref(st)), "qcl_server_wait")
        return self.poll(rid)

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().qcl_server_stats(self.handle, C.byref(s)), "qcl_server_stats")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            load().qcl_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
