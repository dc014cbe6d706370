"""Benchmark: trajectory-steps/s of the FP32-bulk QCL ensemble propagation in
its served form, on the 3-mode ohmic spin-boson workload (1e7 walkers, 2000
steps, outputs every 10 steps), beside the plain FP64 one-launch-per-step
comparator, the FP64 CPU oracle, the other configurations and the served mix.

One timed step = one complete solve submitted to the request server
(qcl_server_submit / qcl_server_wait): model upload, initial Wigner sample,
2000 propagation steps with in-kernel observation every 10 steps, the ensemble
reduction and the copy of the observables to the host.  `value` is measured on
the device (CUDA events the server records on its stream around each busy
period); `e2e` is the host clock around the same calls.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank serves its own 1e7 walkers (global ids
offset by rank), so the per-GPU work is fixed (weak scaling); rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import copy
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2608_14544_gb300 import workloads as wl  # noqa: E402

WORKLOAD = 2
METRIC = ("trajectory-steps/s (FP32-bulk served vs plain FP64) at stated error; "
          "p50/p99 solve latency")
# algorithmic flops of one walker step of a model with more than two states:
# the per-unit figure of the hot-path scope for the four-state Jacobi model
# (300-500 flops), taken at its midpoint
FLOPS_NSTATE = 400.0


def _workload_desc(cfg):
    return (f"3-mode ohmic spin-boson (eps=0.5, Delta=0.5, xi=0.5, wc=2.5, beta=5), "
            f"{cfg['n_traj']:.0e} walkers, dt={cfg['dt']}, {cfg['n_steps']} steps, "
            f"output every {cfg['out_stride']} steps")


def bench_config(cfg, world: int = 1) -> dict:
    """The `config` object of the JSON line (the same in both arms)."""
    return {"workload": _workload_desc(cfg), "n_traj_per_gpu": cfg["n_traj"],
            "n_steps": cfg["n_steps"], "out_stride": cfg["out_stride"],
            "precision": "FP32 bulk, compensated phase/weight, FP64 reduction",
            "l2": "inputs larger than L2 (walker state 460 MB resident in HBM)",
            "parallelism": f"walkers sharded over {world} GPU(s)"}


def flops_per_traj_step(model: dict) -> float:
    """Algorithmic FP32 flops of one walker step, the per-unit figure of the
    hot-path scope.  Two-state models: per mode a drift, the collective
    coordinate sum, a (merged) kick of two FMA and the coupling sum -- 5 FMA =
    10 flops for the spin-boson form, about 12 with the second collective of
    the general two-state form -- plus about 20 scalar FP32 flops and 6 for the
    compensated phase addition (the kernel itself issues 7 FMA per mode, two
    unmerged half kicks, so this count is below the flops it executes).
    Models with more than two states: the scope's four-state figure."""
    if int(model["n_states"]) > 2:
        return FLOPS_NSTATE
    K = np.asarray(model["K"])
    s = 0.5 * (K[:, 0, 0] + K[:, 1, 1])
    b = K[:, 0, 1]
    general = bool(np.any(s != 0) or np.any(b != 0))
    per_mode = 12.0 if general else 10.0
    return per_mode * model["n_modes"] + 26.0


def kernel_source_hash(paths) -> str:
    """sha256 prefix over the kernel's source files (in the given order)."""
    import hashlib

    h = hashlib.sha256()
    for p in paths:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


BULK2_SOURCES = [os.path.join(ROOT, "paper_2608_14544_gb300", "csrc", f)
                 for f in ("kernels_f32.cu", "bulk2.cuh", "lanes.cuh", "qcl_common.cuh",
                           "reduce.cuh", "kernels.h")]


def _profiled(kernel_srcs, summary: str, key: str):
    """A figure from the committed ncu summary (`key: value` line), or None
    when the kernel's sources have changed since the counters were taken."""
    try:
        txt = open(summary).read()
        h = kernel_source_hash(kernel_srcs)
    except OSError:
        return None
    vals = dict(ln.split(":", 1) for ln in txt.splitlines()
                if ln.startswith((key + ":", "traffic_source_sha256_prefix:")))
    if vals.get("traffic_source_sha256_prefix", "").strip() != h or key not in vals:
        return None
    return float(vals[key])


def _profiled_traffic(kernel_srcs, summary: str):
    """DRAM bytes per launch from the committed ncu summary (None if stale)."""
    return _profiled(kernel_srcs, summary, "traffic_bytes_per_launch")


def _issue_roofline(walker_steps_per_s: float, n_sm: int, mhz: float):
    """The kernel is bound by instruction issue: warp instructions per second
    (ncu's instructions per walker-step x the measured rate / 32) against one
    issue per cycle on each of the 4 schedulers of every SM."""
    ipw = _profiled(BULK2_SOURCES, os.path.join(ROOT, "profiles", "k_bulk2_sb3mode.md"),
                    "instructions_per_walker_step")
    if ipw is None:
        return None
    achieved = walker_steps_per_s * ipw / 32.0
    peak = n_sm * 4 * mhz * 1e6
    return {"instructions_per_walker_step": ipw, "achieved_warp_instr_per_s": achieved,
            "peak_warp_instr_per_s": peak, "frac": achieved / peak}


def _result_summary(obs, cfg, status_flags):
    """Observables with their standard errors.  The no-spawn estimator's weights
    grow like exp(2 int |P d/M| dt), so the standard error grows with time; the
    horizon is the last output time at which SE(P_ad) < 0.01."""
    t = np.arange(obs.shape[0]) * cfg["out_stride"] * cfg["dt"]
    ns = int(cfg["model"]["n_states"])
    nq, top = 4 * ns * ns, ns - 1
    ip = 2 * ns * ns + 2 * (top * ns + top)  # the top adiabatic population
    p_ad, se_p = obs[:, ip], obs[:, nq + ip]
    ok = np.where(se_p < 0.01)[0]
    k = int(ok[-1]) if len(ok) else 0
    return {"horizon_t_se_below_0.01": float(t[k]), "P_ad_upper_at_horizon": float(p_ad[k]),
            "se_at_horizon": float(se_p[k]),
            "rho11_minus_rho22_at_horizon": float(obs[k, 0] - obs[k, 2 * (ns + 1)]),
            "trace_at_horizon": float(obs[k, 2 * nq]), "se_P_ad_t_end": float(se_p[-1]),
            "status_flags": status_flags}


def _event_ms(torch, fn, stream=None):
    """CUDA-event time of fn() on the current stream (synchronised both sides)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _request(cfg, n_traj, seed, offset=0):
    return dict(model=cfg["model"], init=cfg["init"], n_traj=int(n_traj), seed=int(seed),
                traj_id_offset=int(offset), n_steps=cfg["n_steps"], dt=cfg["dt"],
                out_stride=cfg["out_stride"])


def spawning_leg(qcl, torch, cfg, n0: int, steps: int, stride: int, capacity_per: int = 64,
                 precisions=(("fp64", 0), ("fp32", 1))):
    """Trajectory spawning (the CPU code's scheme) against the fixed no-spawn
    ensemble of the same initial walkers: the standard error of the upper
    adiabatic population at t = steps dt, the walker-steps each spent, the GPU
    time (CUDA events, sample + propagate), and the products variance x
    walker-steps and variance x seconds (lower is better)."""
    dt = cfg["dt"]
    m = qcl.Model(cfg["model"])
    out = {"workload": f"{cfg['name']} model, {n0} initial walkers, {steps} steps "
                       f"(t = {steps * dt:g})"}
    for name, prec in precisions:
        sp = qcl.SpawnRun(m, n0, capacity_per * n0, cfg["seed"], steps // stride + 1,
                          precision=prec)
        live = []
        t_sp = 0.0
        for rep in range(2):  # the first run warms up
            sp.sample(cfg["init"])
            live = [sp.n_live()]
            ms = 0.0
            for _ in range(steps // stride):
                ms += _event_ms(torch, lambda: sp.propagate(stride, dt, stride))
                live.append(sp.n_live())
            t_sp = ms / 1e3
        ws = float(sum(0.5 * (live[k] + live[k + 1]) * stride for k in range(len(live) - 1)))
        o_s = sp.observables()
        flags = sp.status()["flags"]
        del sp
        ns = qcl.Run(m, n0, cfg["seed"], prec, steps // stride + 1)
        ns.sample(cfg["init"])
        ns.propagate(steps, dt, stride)
        ns.sample(cfg["init"])
        t_ns = _event_ms(torch, lambda: ns.propagate(steps, dt, stride)) / 1e3
        o_n = ns.observables()
        del ns
        ws_ns = float(n0) * steps
        se_s, se_n = float(o_s[-1, 16 + 14]), float(o_n[-1, 16 + 14])
        out[name] = {
            "P_ad_upper": {"spawn": float(o_s[-1, 14]), "no_spawn": float(o_n[-1, 14])},
            "se_P_ad_upper": {"spawn": se_s, "no_spawn": se_n},
            "walker_steps": {"spawn": ws, "no_spawn": ws_ns},
            "final_walkers": live[-1],
            "seconds": {"spawn": t_sp, "no_spawn": t_ns},
            "walker_steps_per_s": {"spawn": ws / t_sp, "no_spawn": ws_ns / t_ns},
            "variance_x_walker_steps": {"spawn": se_s ** 2 * ws, "no_spawn": se_n ** 2 * ws_ns},
            "variance_x_seconds": {"spawn": se_s ** 2 * t_sp, "no_spawn": se_n ** 2 * t_ns},
            "status_flags": flags}
    return out


def stated_error_leg(qcl, torch, cfg, n_nospawn: int, horizons):
    """Error-normalised cost on the benchmark model: for each horizon t, the
    standard error of P_ad(t) and the GPU seconds of a solve to t for the
    FP32-bulk fixed ensemble (no spawning) and for FP32 spawning, and from them
    the seconds either needs to bring SE(P_ad(t)) to 0.01 (variance x seconds /
    1e-4, since the variance falls as 1/walkers and the time grows with
    them)."""
    out = {"model": cfg["name"], "unit": "GPU seconds to SE(P_ad) = 0.01"}
    for t, n0_spawn, cap_per in horizons:
        steps = int(round(t / cfg["dt"]))
        stride = steps
        row = {}
        m = qcl.Model(cfg["model"])
        run = qcl.Run(m, n_nospawn, cfg["seed"], qcl.PREC_FP32_BULK, 2)
        run.sample(cfg["init"])
        run.propagate(steps, cfg["dt"], stride)

        def solve():
            run.sample(cfg["init"])
            run.propagate(steps, cfg["dt"], stride)

        sec = _event_ms(torch, solve) / 1e3
        se = float(run.observables()[-1, 16 + 14])
        row["no_spawn_fp32_bulk"] = {"walkers": n_nospawn, "seconds": sec, "se": se,
                                     "seconds_to_se_0.01": se * se * sec / 1e-4}
        del run
        sp = spawning_leg(qcl, torch, cfg, n0_spawn, steps, stride, capacity_per=cap_per,
                          precisions=(("fp32", 1),))["fp32"]
        if sp["status_flags"] & qcl.FLAG_SPAWN_OVERFLOW:
            row["spawn_fp32"] = {"overflow": True, "initial_walkers": n0_spawn,
                                 "capacity": cap_per * n0_spawn}
        else:
            s_se, s_sec = sp["se_P_ad_upper"]["spawn"], sp["seconds"]["spawn"]
            row["spawn_fp32"] = {"initial_walkers": n0_spawn, "final_walkers": sp["final_walkers"],
                                 "seconds": s_sec, "se": s_se,
                                 "seconds_to_se_0.01": s_se * s_se * s_sec / 1e-4}
        out[f"t={t:g}"] = row
    return out


def ntraj_sweep_leg(qcl, torch, counts, steps: int):
    """Walker-count sweep of the config-2 workload (the paper's statement that
    the time is linear in the number of walkers): per N the CUDA-event time of
    sample + propagate of `steps` steps, after one warm-up solve."""
    cfg = wl.config(2)
    stride, dt = cfg["out_stride"], cfg["dt"]
    m = qcl.Model(cfg["model"])
    m.autotune(dt, stride)
    out = []
    for nt in counts:
        run = qcl.Run(m, int(nt), cfg["seed"], qcl.PREC_FP32_BULK, steps // stride + 1)
        run.sample(cfg["init"])
        run.propagate(steps, dt, stride)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        run.sample(cfg["init"])
        run.propagate(steps, dt, stride)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out.append({"n_traj": int(nt), "ms": ms, "walker_steps_per_s": nt * steps / (ms / 1e3),
                    "ns_per_walker_step": ms * 1e6 / (nt * steps)})
        del run
    return {"workload": f"config-2 model, {steps} steps per point, FP32 bulk (sample + propagate)",
            "points": out}



def served_mix_leg(qcl, reqs, arena_gb: float, quantum: int, paced: bool, peak_tflops: float,
                   round_flops: float = 0.0):
    """Requests replayed against the server, either at their Poisson arrival
    times (paced) or all at once (saturating), with every request advancing a
    quantum per round (round_flops = 0) or the shortest remaining work first
    under a round budget: per-request latency (finish - submit) percentiles,
    aggregate trajectory-steps/s over the host span and over the device's busy
    time, and the algorithmic FP32 flops of all requests against the FP32 peak
    (the fraction of the roofline the mix reaches)."""
    srv = qcl.Server(int(arena_gb * (1 << 30)), max_active=256, quantum_steps=quantum,
                     round_flops=round_flops)
    t0 = time.perf_counter()
    ids = []
    for r in reqs:
        if paced:
            dt_wait = t0 + r["arrival_s"] - time.perf_counter()
            if dt_wait > 0:
                time.sleep(dt_wait)
        ids.append(srv.submit(r))
    errors = 0
    for rid in ids:
        st, _ = srv.wait(rid, 3600.0)
        errors += st != qcl.REQ_DONE
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    kinds = [0] * 5
    flops = 0.0
    for r in reqs:
        kinds[r["kind"]] += 1
        flops += float(r["n_traj"]) * r["n_steps"] * flops_per_traj_step(r["model"])
    dev = st["device_busy_s"]
    achieved = flops / dev / 1e12 if dev > 0 else None
    return {"requests": len(reqs), "arrivals": "Poisson, mean gap 5 ms" if paced else "all at t = 0",
            "scheduling": (f"shortest remaining work first, {round_flops:.0e} flops per round"
                           if round_flops > 0 else "every active request a quantum per round"),
            "kinds_sb1_sb3_vib3_sb100_lvc4": kinds,
            "n_traj_range": [min(r["n_traj"] for r in reqs), max(r["n_traj"] for r in reqs)],
            "traj_steps": sum(float(r["n_traj"]) * r["n_steps"] for r in reqs),
            "latency_p50_s": st["latency_p50_s"], "latency_p99_s": st["latency_p99_s"],
            "latency_mean_s": st["latency_mean_s"], "throughput": st["throughput"],
            "device_busy_s": dev, "device_throughput": st["device_throughput"],
            "unit": "traj-steps/s", "span_s": st["span_s"], "wall_s": wall,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved / peak_tflops if achieved else None,
                         "basis": "algorithmic flops of every request over the device busy time"},
            "rounds": st["rounds"], "graph_replays": st["graph_replays"],
            "errors": int(errors + st["n_error"]), "quantum_steps": quantum}


def config_leg(qcl, torch, cfg, n_traj: int, stream, peak_tflops: float, probe_steps=None,
               counted: bool = True):
    """One full-size solve of a configuration through the single-solve entry
    points (sample + propagate + device reduction), after a short warm-up run
    of the same kernels: walker-steps/s, and the dominant kernel's algorithmic
    FP32 flops against the FP32 peak (counted = False: no per-unit flop figure
    applies, the rate alone)."""
    stride, dt, steps = cfg["out_stride"], cfg["dt"], cfg["n_steps"]
    m = qcl.Model(cfg["model"])
    shape = m.autotune(dt, stride, probe_walkers=1 << 20,
                       n_steps=probe_steps or 32 * stride)
    n_out = steps // stride + 1
    run = qcl.Run(m, n_traj, cfg["seed"], qcl.PREC_FP32_BULK, n_out)
    dev = torch.empty((n_out, 2 * 4 * cfg["model"]["n_states"] ** 2 + 3), dtype=torch.float64,
                      device="cuda")
    run.sample(cfg["init"])
    run.propagate(min(steps, 32 * stride), dt, stride)
    qcl.kernel_time(qcl.KERNEL_BULK)
    qcl.set_option(qcl.OPT_TIMING, 1)

    def solve():
        run.sample(cfg["init"])
        run.step = 0
        run.propagate(steps, dt, stride)
        run.observables_device(dev)

    ms = _event_ms(torch, solve, stream)
    qcl.set_option(qcl.OPT_TIMING, 0)
    k_ms, k_n = qcl.kernel_time(qcl.KERNEL_BULK)
    fl = flops_per_traj_step(cfg["model"]) if counted else None
    ach = float(n_traj) * steps * fl / (k_ms / 1e3) / 1e12 if (k_ms > 0 and fl) else None
    flags = run.status()["flags"]
    obs = dev.cpu().numpy()
    del run
    return {"n_traj": n_traj, "n_steps": steps, "dt": dt, "out_stride": stride,
            "value": float(n_traj) * steps / (ms / 1e3), "unit": "traj-steps/s",
            "ms_per_solve": ms, "launch_shape": shape, "flops_per_traj_step": fl,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": ach / peak_tflops if ach else None,
                         "kernel_ms_per_launch": k_ms / max(k_n, 1), "launches": k_n},
            "result": _result_summary(obs, cfg, flags)}


# ------------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[4 + k].lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle --
def cpu_oracle_rate(cfg, target_s: float, threads: int):
    """The FP64 oracle as it stands on the host cores: a bounded sample of the
    same workload (all steps, fewer walkers), trajectory-steps/s."""
    import oracle

    oracle.build()
    om = oracle.OracleModel(cfg["model"])
    oi = oracle.OracleInit(om, cfg["init"])
    steps = cfg["n_steps"]
    t0 = time.perf_counter()
    probe = 64
    oracle.run(om, oi, cfg["seed"], 0, probe, cfg["dt"], steps, cfg["out_stride"])
    per_walker = (time.perf_counter() - t0) / probe
    n = max(threads, int(target_s * threads / max(per_walker, 1e-9)))
    t0 = time.perf_counter()
    oracle.run_threaded(om, oi, cfg["seed"], n, cfg["dt"], steps, cfg["out_stride"], threads)
    el = time.perf_counter() - t0
    return n * steps / el, n, el


# ---------------------------------------------------------------- reference --
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = wl.config(WORKLOAD)
    threads = os.cpu_count() or 1
    import oracle

    oracle.build()
    om = oracle.OracleModel(cfg["model"])
    oi = oracle.OracleInit(om, cfg["init"])
    steps = cfg["n_steps"]
    # size one step to about 4 s of host work
    t0 = time.perf_counter()
    oracle.run(om, oi, 0, 0, 32, cfg["dt"], steps, cfg["out_stride"])
    per_walker = (time.perf_counter() - t0) / 32
    n = max(threads, int(4.0 * threads / max(per_walker, 1e-9)))
    for _ in range(args.warmup):
        oracle.run_threaded(om, oi, cfg["seed"], n, cfg["dt"], steps, cfg["out_stride"], threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run_threaded(om, oi, cfg["seed"], n, cfg["dt"], steps, cfg["out_stride"], threads)
    el = time.perf_counter() - t0
    value = n * steps * args.steps / el
    sample = (f"{n} walkers x {steps} steps per timed step (of {cfg['n_traj']:.0e} walkers), "
              f"FP64 oracle on {threads} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "traj-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(cfg, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": "traj-steps/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "traj-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------- ours --
def run_ours(args):
    import torch

    from paper_2608_14544_gb300 import build as qbuild
    from paper_2608_14544_gb300 import qcl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        qbuild.build()
    if dist:
        dist.barrier()
    qcl.load()

    def max_over_ranks(x: float) -> float:
        if not dist:
            return x
        t = torch.tensor([x], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    cfg = wl.config(WORKLOAD)
    n, steps, stride, dt = cfg["n_traj"], cfg["n_steps"], cfg["out_stride"], cfg["dt"]
    n_out = steps // stride + 1
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(0)
    n_sm = props.multi_processor_count
    max_mhz = 2070.0
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        max_mhz = float(json.load(open(peaks_path)).get("sm_max_mhz", max_mhz))
    peak_tflops = n_sm * 128 * 2 * max_mhz * 1e6 / 1e12
    fl = flops_per_traj_step(cfg["model"])

    # ---- the served form (headline): one solve per step through the server
    req = _request(cfg, n, cfg["seed"], offset=rank * n)
    m = cfg["model"]
    h2d = sum(np.asarray(m[k], dtype=np.float64).nbytes for k in ("mass", "omega", "E", "K"))
    h2d += sum(np.asarray(cfg["init"][k], dtype=np.float64).nbytes for k in ("rho_el0", "R0", "P0"))
    srv = qcl.Server(4 << 30, max_active=4, quantum_steps=args.headline_quantum)
    for _ in range(max(args.warmup, 0)):
        srv.wait(srv.submit(req))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    s0 = srv.stats()
    qcl.launch_count(reset=True)
    qcl.kernel_time(qcl.KERNEL_BULK)
    qcl.set_option(qcl.OPT_TIMING, 1)
    solve_s = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            t1 = time.perf_counter()
            st, host_obs = srv.wait(srv.submit(req))
            solve_s.append(time.perf_counter() - t1)
            if st != qcl.REQ_DONE:
                raise RuntimeError("served solve failed")
        torch.cuda.synchronize()
        host_s = time.perf_counter() - t0
    qcl.set_option(qcl.OPT_TIMING, 0)
    launches = qcl.launch_count()
    bulk_ms, bulk_n = qcl.kernel_time(qcl.KERNEL_BULK)
    s1 = srv.stats()
    srv.close()
    dev_s = max_over_ranks(s1["device_busy_s"] - s0["device_busy_s"])
    host_s = max_over_ranks(host_s)
    traj_steps = float(n) * steps * args.steps * world
    value = traj_steps / dev_s
    achieved = float(n) * steps * args.steps * fl / (bulk_ms / 1e3) / 1e12 if bulk_ms > 0 else None
    e2e = {"value": traj_steps / host_s, "unit": "traj-steps/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(host_obs.nbytes),
           "path": "qcl_server_submit / qcl_server_wait / qcl_server_poll (host descriptors in, "
                   "host observables out), host clock"}

    # ---- the same solve through the single-solve entry points
    model = qcl.Model(cfg["model"])
    shape = model.autotune(dt, stride)
    run = qcl.Run(model, n, cfg["seed"], qcl.PREC_FP32_BULK, n_out, traj_id_offset=rank * n)
    dev_obs = torch.empty((n_out, 8 * 4 + 3), dtype=torch.float64, device="cuda")

    def solve():
        run.sample(cfg["init"])
        run.step = 0
        run.propagate(steps, dt, stride)
        run.observables_device(dev_obs)

    for _ in range(max(args.warmup, 0)):
        solve()
    qcl.kernel_time(qcl.KERNEL_BULK)
    qcl.set_option(qcl.OPT_TIMING, 1)
    d_ms = _event_ms(torch, lambda: [solve() for _ in range(args.steps)], stream)
    qcl.set_option(qcl.OPT_TIMING, 0)
    dk_ms, dk_n = qcl.kernel_time(qcl.KERNEL_BULK)
    d_ach = float(n) * steps * args.steps * fl / (dk_ms / 1e3) / 1e12 if dk_ms > 0 else None
    direct = {"value": float(n) * steps * args.steps / (d_ms / 1e3), "unit": "traj-steps/s",
              "ms_per_solve": d_ms / args.steps, "launch_shape": shape,
              "path": "qcl_sample_initial / qcl_propagate / qcl_finalize_observables, CUDA events",
              "roofline": {"bound": "alu", "achieved": d_ach, "peak": peak_tflops, "unit": "TFLOP/s",
                           "frac": d_ach / peak_tflops if d_ach else None,
                           "kernel_ms_per_launch": dk_ms / max(dk_n, 1), "launches": dk_n}}
    del run

    # ---- FP64 comparator: the paper's structure (one launch per step, SoA in
    # HBM), same walkers, a bounded number of steps
    fp64_steps = 100
    run64 = qcl.Run(model, n, cfg["seed"], qcl.PREC_FP64, fp64_steps // stride + 1,
                    traj_id_offset=rank * n)
    run64.sample(cfg["init"])
    run64.propagate(stride, dt, stride)
    qcl.kernel_time(qcl.KERNEL_FP64_STEP)
    qcl.set_option(qcl.OPT_TIMING, 1)
    f_ms = _event_ms(torch, lambda: run64.propagate(fp64_steps - stride, dt, stride), stream)
    qcl.set_option(qcl.OPT_TIMING, 0)
    f64_ms, f64_n = qcl.kernel_time(qcl.KERNEL_FP64_STEP)
    fp64_rate = float(n) * (fp64_steps - stride) / (f_ms / 1e3)
    del run64

    legs = {}
    # ---- the other configurations at their stated sizes
    if args.cfg3_walkers > 0:
        legs["vibronic3"] = dict(config_leg(qcl, torch, wl.config(3), args.cfg3_walkers, stream,
                                            peak_tflops),
                                 workload="synthetic 2-state 3-mode LVC model with a conical "
                                          "intersection (eV/fs), ground Wigner in S2")
    if args.sb100_walkers > 0:
        legs["sb100"] = dict(config_leg(qcl, torch, wl.config(4), args.sb100_walkers, stream,
                                        peak_tflops),
                             workload="100-mode ohmic spin-boson (eps=Delta=1, xi=0.25, wc=5, "
                                      "beta=1)")
    if args.sb100_walkers > 0:
        c4d = copy.deepcopy(wl.config(4))
        c4d["model"]["repr"] = "diabatic"
        legs["sb100_diabatic"] = dict(
            config_leg(qcl, torch, c4d, args.sb100_walkers, stream, peak_tflops, counted=False),
            workload="the 100-mode model in the diabatic representation (the split kernel's "
                     "diabatic form; no per-unit flop figure in the scope)")
    cd = copy.deepcopy(cfg)
    cd["model"]["repr"] = "diabatic"
    legs["diabatic"] = dict(config_leg(qcl, torch, cd, n, stream, peak_tflops),
                            workload="the benchmark solve in the diabatic representation")
    if args.nstate_walkers > 0:
        c4 = wl.lvc4_config(1)
        legs["lvc4"] = dict(config_leg(qcl, torch, c4, args.nstate_walkers, stream, peak_tflops),
                            workload="random four-state six-mode LVC model (the served mix's "
                                     "four-state kind), 1000 steps, outputs every 10")
        c4d = copy.deepcopy(c4)
        c4d["model"]["repr"] = "diabatic"
        legs["lvc4_diabatic"] = dict(
            config_leg(qcl, torch, c4d, args.nstate_walkers, stream, peak_tflops, counted=False),
            workload="the same model in the diabatic representation (no decomposition in the "
                     "step; no per-unit flop figure in the scope)")
        c64 = wl.lvc4_config(1, 64)
        legs["lvc4_64modes"] = dict(
            config_leg(qcl, torch, c64, args.nstate_walkers, stream, peak_tflops, counted=False),
            workload="random four-state 64-mode LVC model (R and P kept in the ensemble buffer "
                     "by the modes-in-memory kernel), 1000 steps, outputs every 10")
    if args.spawn_walkers > 0:
        legs["spawning"] = spawning_leg(qcl, torch, wl.config(1), args.spawn_walkers, 400, 20)
        # (horizon, initial spawning walkers, slots per initial walker): the
        # spawned population grows about 30-fold by t = 1.6 on this model
        legs["stated_error"] = stated_error_leg(
            qcl, torch, cfg, n, ((1.6, args.stated_spawn_walkers, 256),
                                 (4.0, max(args.stated_spawn_walkers // 10, 1), 16384)))
    if args.ntraj_sweep and rank == 0:
        legs["ntraj_sweep"] = ntraj_sweep_leg(qcl, torch, [1e4, 1e5, 1e6, 1e7, 1e8], 400)
    if args.served_requests > 0 and rank == 0:
        reqs = wl.served_mix(n_requests=args.served_requests, traj_range=(1e4, args.served_traj_max))
        legs["served_mix"] = {
            "paced": served_mix_leg(qcl, reqs, args.served_arena_gb, args.served_quantum, True,
                                    peak_tflops),
            "paced_shortest_first": served_mix_leg(qcl, reqs, args.served_arena_gb,
                                                   args.served_quantum, True, peak_tflops,
                                                   args.served_round_flops),
            "saturating_shortest_first": served_mix_leg(qcl, reqs, args.served_arena_gb,
                                                        args.served_quantum, False, peak_tflops,
                                                        args.served_round_flops)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # our own FMA microbenchmarks beside the derived peak (FP32 FFMA for the bulk
    # kernels, FP64 DFMA for the comparator)
    peak_fp32_meas = qcl.measure_peak(0) / 1e12
    peak_fp64_meas = qcl.measure_peak(1) / 1e12
    clocks = clk.summary()
    cpu_threads = os.cpu_count() or 1
    cpu_rate, cpu_n, cpu_s = cpu_oracle_rate(cfg, args.cpu_seconds, cpu_threads)
    cpu1_rate, cpu1_n, cpu1_s = cpu_oracle_rate(cfg, args.cpu_seconds / 3, 1)
    lat = np.array(solve_s)
    out = {
        "metric": METRIC, "value": value, "unit": "traj-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": bench_config(cfg, world),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": (achieved / peak_tflops) if achieved else None,
                     "traffic": _profiled_traffic(
                         BULK2_SOURCES, os.path.join(ROOT, "profiles", "k_bulk2_sb3mode.md")),
                     "traffic_unit": "DRAM bytes per launch (ncu, 4M-walker launch scaled)",
                     "kernel": "k_bulk2 (persistent FP32-bulk walker kernel)",
                     "flops_per_traj_step": fl,
                     "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {max_mhz:.0f} MHz",
                     "peak_microbench_tflops": {"fp32_ffma": peak_fp32_meas,
                                                "fp64_dfma": peak_fp64_meas},
                     "issue_slots": _issue_roofline(value / world, n_sm, max_mhz),
                     "kernel_ms_per_launch": bulk_ms / max(bulk_n, 1), "launches": bulk_n},
        "cpu_baseline": {"value": cpu_rate, "unit": "traj-steps/s", "cores": cpu_threads,
                         "kind": "oracle",
                         "sample": f"{cpu_n} walkers x {steps} steps of the same workload "
                                   f"({cpu_s:.1f} s)",
                         "single_thread": {"value": cpu1_rate, "cores": 1,
                                           "sample": f"{cpu1_n} walkers x {steps} steps "
                                                     f"({cpu1_s:.1f} s)"}},
        "e2e": e2e,
        "gpu_launches": launches,
        "served": {"path": "qcl_server_submit / qcl_server_wait, one 1e7-walker request per step",
                   "device_ms_per_solve": 1e3 * dev_s / args.steps,
                   "host_ms_per_solve": 1e3 * host_s / args.steps,
                   "solve_latency_p50_s": float(np.percentile(lat, 50)),
                   "solve_latency_p99_s": float(np.percentile(lat, 99)),
                   "rounds_per_solve": (s1["rounds"] - s0["rounds"]) / args.steps,
                   "timing": "value: CUDA events on the server stream around each busy period "
                             "(sampling to retirement); e2e: host clock"},
        "direct": direct,
        "fp64_comparator": {"value": fp64_rate, "unit": "traj-steps/s",
                            "sample": f"{n:.0e} walkers x {fp64_steps - stride} steps, one "
                                      "launch per step", "step_kernel_ms": f64_ms / max(f64_n, 1),
                            "speedup_of_fp32_bulk_served": value / world / fp64_rate,
                            "frac_of_fp64_dfma_peak": fp64_rate * fl / 1e12 / peak_fp64_meas
                            if peak_fp64_meas > 0 else None},
        **legs,
        "clocks": clocks,
        "result": _result_summary(host_obs, cfg, 0),
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--headline-quantum", type=int, default=2000)
    ap.add_argument("--cfg3-walkers", type=int, default=100_000_000)
    ap.add_argument("--sb100-walkers", type=int, default=10_000_000)
    ap.add_argument("--spawn-walkers", type=int, default=100_000)
    ap.add_argument("--stated-spawn-walkers", type=int, default=20_000)
    ap.add_argument("--ntraj-sweep", type=int, default=1, help="0 skips the walker-count sweep")
    ap.add_argument("--served-requests", type=int, default=256)
    ap.add_argument("--served-traj-max", type=float, default=1e7)
    ap.add_argument("--served-arena-gb", type=float, default=128.0)
    ap.add_argument("--served-quantum", type=int, default=400)
    ap.add_argument("--nstate-walkers", type=int, default=4_000_000,
                    help="walkers of the four-state legs (0: skip)")
    ap.add_argument("--served-round-flops", type=float, default=2e12,
                    help="round work budget of the shortest-first served-mix legs")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
