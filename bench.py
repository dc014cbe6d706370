"""Benchmark: trajectory-steps/s of the FP32-bulk QCL ensemble propagation on
the 3-mode ohmic spin-boson workload (1e7 walkers, 2000 steps), beside the
FP64 one-launch-per-step comparator and the CPU FP64 oracle.

One timed step = one complete solve: initial Wigner sample, 2000 propagation
steps with in-kernel observation every 10 steps, and the ensemble reduction.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank propagates its own 1e7 walkers (global ids
offset by rank), so the per-GPU work is fixed (weak scaling); rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
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
METRIC = "trajectory-steps/s (FP32-bulk, served form) at stated error"


def _workload_desc(cfg):
    return (f"3-mode ohmic spin-boson (eps=0.5, Delta=0.5, xi=0.5, wc=2.5, beta=5), "
            f"{cfg['n_traj']:.0e} walkers, dt={cfg['dt']}, {cfg['n_steps']} steps, "
            f"output every {cfg['out_stride']} steps")


def flops_per_traj_step(model: dict) -> float:
    """Algorithmic FP32 flops of one walker step of a two-state model, the
    per-unit figure of the hot-path scope: per mode a drift, the collective
    coordinate sum, a (merged) kick of two FMA and the coupling sum -- 5 FMA =
    10 flops for the spin-boson form, about 12 with the second collective of
    the general two-state form -- plus about 20 scalar FP32 flops and 6 for the
    compensated phase addition.  The kernel itself issues 7 FMA per mode (two
    unmerged half kicks, see the kernel notes), so this count is below the
    flops it executes."""
    K = model["K"]
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


def _result_summary(obs, cfg, status):
    """Observables with their standard errors.  The no-spawn estimator's weights
    grow like exp(2 int |P d/M| dt), so the standard error grows with time; the
    horizon is the last output time at which SE(P_ad) < 0.01."""
    t = np.arange(obs.shape[0]) * cfg["out_stride"] * cfg["dt"]
    p_ad, se_p = obs[:, 14], obs[:, 16 + 14]
    ok = np.where(se_p < 0.01)[0]
    k = int(ok[-1]) if len(ok) else 0
    return {"horizon_t_se_below_0.01": float(t[k]), "P_ad_upper_at_horizon": float(p_ad[k]),
            "se_at_horizon": float(se_p[k]),
            "rho11_minus_rho22_at_horizon": float(obs[k, 0] - obs[k, 6]),
            "trace_at_horizon": float(obs[k, 32]), "se_P_ad_t_end": float(se_p[-1]),
            "status_flags": status["flags"]}


def spawning_leg(qcl, torch, n0: int, steps: int, stride: int):
    """Trajectory spawning (the CPU code's scheme) against the fixed no-spawn
    ensemble on the 1-mode spin-boson model, in FP64 and in FP32 bulk: the
    standard error of the upper adiabatic population at t = steps dt, the
    walker-steps each spent, the GPU time (CUDA events, sample + propagate), and
    the products variance x walker-steps and variance x seconds (lower is
    better).  Same seed for all four."""
    cfg = wl.config(1)
    dt = cfg["dt"]
    m = qcl.Model(cfg["model"])
    out = {"workload": f"1-mode spin-boson (cfg 1 model), {n0} initial walkers, {steps} steps "
                       f"(t = {steps * dt:g})"}
    for name, prec in (("fp64", qcl.PREC_FP64), ("fp32", qcl.PREC_FP32_BULK)):
        sp = qcl.SpawnRun(m, n0, 64 * n0, cfg["seed"], steps // stride + 1, precision=prec)
        live = []
        t_sp = 0.0
        for rep in range(2):  # the first run warms up
            sp.sample(cfg["init"])
            live = [sp.n_live()]
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            ms = 0.0
            for _ in range(steps // stride):
                e0.record()
                sp.propagate(stride, dt, stride)
                e1.record()
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
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
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ns.propagate(steps, dt, stride)
        e1.record()
        torch.cuda.synchronize()
        t_ns = e0.elapsed_time(e1) / 1e3
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


def served_mix_leg(qcl, n_requests: int, traj_hi: float, arena_gb: float, quantum: int):
    """Poisson-arriving requests (mean gap 5 ms) drawn uniformly from the
    1-mode, 3-mode, 3-mode vibronic and 100-mode models and a random 4-state
    model, replayed in real time against the server: per-request latency
    (finish - submit) percentiles and aggregate trajectory-steps/s."""
    reqs = wl.served_mix(n_requests=n_requests, traj_range=(1e4, traj_hi))
    srv = qcl.Server(int(arena_gb * (1 << 30)), max_active=256, quantum_steps=quantum)
    t0 = time.perf_counter()
    ids = []
    for r in reqs:
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
    for r in reqs:
        kinds[r["kind"]] += 1
    return {"requests": n_requests, "kinds_sb1_sb3_vib3_sb100_lvc4": kinds,
            "n_traj_range": [1e4, traj_hi], "steps_range": [500, 4000],
            "latency_p50_s": st["latency_p50_s"], "latency_p99_s": st["latency_p99_s"],
            "latency_mean_s": st["latency_mean_s"], "throughput": st["throughput"],
            "unit": "traj-steps/s", "span_s": st["span_s"], "wall_s": wall,
            "rounds": st["rounds"], "graph_replays": st["graph_replays"],
            "errors": int(errors + st["n_error"]), "quantum_steps": quantum}


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
    sample = f"{n} walkers x {steps} steps per timed step (of {cfg['n_traj']:.0e} walkers)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "traj-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_desc(cfg), "n_traj_sampled": n},
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

    cfg = wl.config(WORKLOAD)
    n, steps, stride, dt = cfg["n_traj"], cfg["n_steps"], cfg["out_stride"], cfg["dt"]
    n_out = steps // stride + 1
    model = qcl.Model(cfg["model"])
    # launch shape (walkers per thread, blocks per SM) picked by the library's
    # autotuner on a probe ensemble -- setup, outside every timed region
    shape = model.autotune(dt, stride)
    run = qcl.Run(model, n, cfg["seed"], qcl.PREC_FP32_BULK, n_out, traj_id_offset=rank * n)
    stream = torch.cuda.current_stream()

    # means and standard errors of every output time, finalised on the device
    dev_obs = torch.empty((n_out, 8 * 4 + 3), dtype=torch.float64, device="cuda")

    def solve():
        run.sample(cfg["init"])
        run.propagate(steps, dt, stride)
        # ensemble reduction into the device rows is part of propagate; the
        # finalisation of means/SE runs on the device into dev_obs (the timed
        # region has no host synchronisation; the end-to-end figure below reads
        # the results back every step)
        run.observables_device(dev_obs)

    for _ in range(max(args.warmup, 0)):
        solve()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    qcl.launch_count(reset=True)
    qcl.kernel_time(qcl.KERNEL_BULK)
    qcl.set_option(qcl.OPT_TIMING, 1)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            solve()
        ev1.record(stream)
        torch.cuda.synchronize()
    obs = dev_obs.cpu().numpy()
    qcl.set_option(qcl.OPT_TIMING, 0)
    launches = qcl.launch_count()
    bulk_ms, bulk_n = qcl.kernel_time(qcl.KERNEL_BULK)
    el_ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([el_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el_ms = float(t.item())
    traj_steps = float(n) * steps * args.steps * world
    value = traj_steps / (el_ms / 1e3)
    status = run.status()

    # FP64 comparator: the paper's structure (one launch per step, SoA in HBM),
    # same walkers, a bounded number of steps
    fp64_steps = 100
    run64 = qcl.Run(model, n, cfg["seed"], qcl.PREC_FP64, fp64_steps // stride + 1,
                    traj_id_offset=rank * n)
    run64.sample(cfg["init"])
    run64.propagate(stride, dt, stride)
    torch.cuda.synchronize()
    qcl.kernel_time(qcl.KERNEL_FP64_STEP)
    qcl.set_option(qcl.OPT_TIMING, 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run64.propagate(fp64_steps - stride, dt, stride)
    e1.record(stream)
    torch.cuda.synchronize()
    qcl.set_option(qcl.OPT_TIMING, 0)
    f64_ms, f64_n = qcl.kernel_time(qcl.KERNEL_FP64_STEP)
    fp64_rate = float(n) * (fp64_steps - stride) / (e0.elapsed_time(e1) / 1e3)
    del run64

    # end to end through the C ABI with host buffers: model upload, sample,
    # propagate, device reduction and the copy of the observables to the host
    m = cfg["model"]
    h2d = sum(np.asarray(m[k], dtype=np.float64).nbytes for k in ("mass", "omega", "E", "K"))
    h2d += sum(np.asarray(cfg["init"][k], dtype=np.float64).nbytes for k in ("rho_el0", "R0", "P0"))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mm = qcl.Model(m)
        mm.set_launch_shape(shape["walkers_per_thread"], shape["blocks_per_sm"])
        rr = qcl.Run(mm, n, cfg["seed"], qcl.PREC_FP32_BULK, n_out, traj_id_offset=rank * n)
        rr.sample(cfg["init"])
        rr.propagate(steps, dt, stride)
        host_obs = rr.observables()
        del rr
        mm.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": traj_steps / e2e_s, "unit": "traj-steps/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(host_obs.nbytes)}

    # many-mode workload (100-mode ohmic spin-boson, the configuration where the
    # FP32 FMA work dominates): bounded walker count, all 4000 steps
    c4 = wl.config(4)
    n4 = args.sb100_walkers
    m4 = qcl.Model(c4["model"])
    # (probe: 2^20 walkers over one full persistent launch of 32 outputs; a
    # short probe of 40 steps favoured one walker per thread, which is slower
    # at 2e6 walkers x 4000 steps)
    shape4 = m4.autotune(c4["dt"], c4["out_stride"], probe_walkers=1 << 20,
                         n_steps=32 * c4["out_stride"])
    r4 = qcl.Run(m4, n4, c4["seed"], qcl.PREC_FP32_BULK, c4["n_steps"] // c4["out_stride"] + 1,
                 traj_id_offset=rank * n4)
    r4.sample(c4["init"])
    r4.propagate(c4["n_steps"], c4["dt"], c4["out_stride"])
    torch.cuda.synchronize()
    r4.sample(c4["init"])
    qcl.kernel_time(qcl.KERNEL_BULK)
    qcl.set_option(qcl.OPT_TIMING, 1)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    r4.propagate(c4["n_steps"], c4["dt"], c4["out_stride"])
    g1.record(stream)
    torch.cuda.synchronize()
    qcl.set_option(qcl.OPT_TIMING, 0)
    k4_ms, k4_n = qcl.kernel_time(qcl.KERNEL_BULK)
    rate4 = float(n4) * c4["n_steps"] / (g0.elapsed_time(g1) / 1e3)
    st4 = r4.status()
    del r4

    # the same 3-mode workload in the diabatic representation (one solve after a
    # warm-up solve; the walkers' state is the same size, the step is shorter:
    # no per-step decomposition)
    import copy

    cd = copy.deepcopy(cfg)
    cd["model"]["repr"] = "diabatic"
    md = qcl.Model(cd["model"])
    md.autotune(dt, stride)
    rd = qcl.Run(md, n, cfg["seed"], qcl.PREC_FP32_BULK, n_out, traj_id_offset=rank * n)
    rd.sample(cd["init"])
    rd.propagate(steps, dt, stride)
    rd.sample(cd["init"])
    torch.cuda.synchronize()
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    rd.propagate(steps, dt, stride)
    h1.record(stream)
    torch.cuda.synchronize()
    rate_dia = float(n) * steps / (h0.elapsed_time(h1) / 1e3)
    std = rd.status()
    del rd

    spawning = spawning_leg(qcl, torch, args.spawn_walkers, 400, 20) if args.spawn_walkers > 0 \
        else None
    sweep = ntraj_sweep_leg(qcl, torch, [1e4, 1e5, 1e6, 1e7, 1e8], 400) \
        if (args.ntraj_sweep and rank == 0) else None

    served = None
    if args.served_requests > 0 and rank == 0:
        served = served_mix_leg(qcl, args.served_requests, args.served_traj_max,
                                args.served_arena_gb, args.served_quantum)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # our own FMA microbenchmarks beside the derived peak (FP32 FFMA for the bulk
    # kernels, FP64 DFMA for the comparator)
    peak_fp32_meas = qcl.measure_peak(0) / 1e12
    peak_fp64_meas = qcl.measure_peak(1) / 1e12

    # roofline of the dominant kernel (FP32 ALU bound)
    props = torch.cuda.get_device_properties(0)
    n_sm = props.multi_processor_count
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    max_mhz = 2070.0
    if os.path.exists(peaks_path):
        max_mhz = float(json.load(open(peaks_path)).get("sm_max_mhz", max_mhz))
    clocks = clk.summary()
    if clocks and clocks.get("sm_max_mhz"):
        max_mhz = clocks["sm_max_mhz"]
    peak_tflops = n_sm * 128 * 2 * max_mhz * 1e6 / 1e12
    fl = flops_per_traj_step(m)
    achieved = float(n) * steps * args.steps * fl / (bulk_ms / 1e3) / 1e12 if bulk_ms > 0 else None
    cpu_threads = os.cpu_count() or 1
    cpu_rate, cpu_n, cpu_s = cpu_oracle_rate(cfg, args.cpu_seconds, cpu_threads)

    mean = obs[:, :16]
    out = {
        "metric": METRIC, "value": value, "unit": "traj-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": _workload_desc(cfg), "n_traj_per_gpu": n, "n_steps": steps,
                   "out_stride": stride, "precision": "FP32 bulk, compensated phase/weight, "
                   "FP64 reduction", "l2": "inputs larger than L2 (walker state "
                   f"{qcl.ensemble_bytes(model, run.ens) / 1e6:.0f} MB resident in HBM)",
                   "parallelism": f"walkers sharded over {world} GPU(s)",
                   "launch_shape": shape},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": (achieved / peak_tflops) if achieved else None,
                     "traffic": _profiled_traffic(
                         BULK2_SOURCES, os.path.join(ROOT, "profiles", "k_bulk2_sb3mode.md")),
                     "traffic_unit": "bytes per launch (ncu, small case scaled)",
                     "kernel": "k_bulk2 (persistent FP32-bulk walker kernel)",
                     "flops_per_traj_step": fl,
                     "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {max_mhz:.0f} MHz",
                     "peak_microbench_tflops": {"fp32_ffma": peak_fp32_meas,
                                                "fp64_dfma": peak_fp64_meas},
                     "issue_slots": _issue_roofline(value / world, n_sm, max_mhz),
                     "kernel_ms_per_launch": bulk_ms / max(bulk_n, 1),
                     "launches": bulk_n},
        "cpu_baseline": {"value": cpu_rate, "unit": "traj-steps/s", "cores": cpu_threads,
                         "kind": "oracle",
                         "sample": f"{cpu_n} walkers x {steps} steps of the same workload "
                                   f"({cpu_s:.1f} s)"},
        "e2e": e2e,
        "gpu_launches": launches,
        "fp64_comparator": {"value": fp64_rate, "unit": "traj-steps/s",
                            "sample": f"{n:.0e} walkers x {fp64_steps - stride} steps, one "
                                      "launch per step", "step_kernel_ms": f64_ms / max(f64_n, 1),
                            "speedup_of_fp32_bulk": value / world / fp64_rate,
                            "frac_of_fp64_dfma_peak": fp64_rate * fl / 1e12 / peak_fp64_meas
                            if peak_fp64_meas > 0 else None},
        "sb100": {"workload": f"100-mode ohmic spin-boson (eps=Delta=1, xi=0.25, wc=5, beta=1), "
                              f"{n4} walkers x {c4['n_steps']} steps, dt={c4['dt']}",
                  "value": rate4, "unit": "traj-steps/s",
                  "flops_per_traj_step": flops_per_traj_step(c4["model"]),
                  "achieved_tflops": float(n4) * c4["n_steps"] * flops_per_traj_step(c4["model"])
                  / (k4_ms / 1e3) / 1e12 if k4_ms > 0 else None,
                  "frac_of_fp32_peak": (float(n4) * c4["n_steps"] * flops_per_traj_step(c4["model"])
                                        / (k4_ms / 1e3) / 1e12 / peak_tflops) if k4_ms > 0 else None,
                  "kernel": "k_bulk2_split2 (four warps per 32 walker slots, two walkers per "
                            "thread)", "launch_shape": shape4,
                  "status_flags": st4["flags"]},
        "diabatic": {"workload": "the same 3-mode spin-boson solve in the diabatic "
                                 "representation (propagation only)",
                     "value": rate_dia, "unit": "traj-steps/s", "kernel": "k_bulk2_dia",
                     "status_flags": std["flags"]},
        "spawning": spawning,
        "ntraj_sweep": sweep,
        "served_mix": served,
        "clocks": clocks,
        "result": _result_summary(obs, cfg, status),
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
    ap.add_argument("--sb100-walkers", type=int, default=2_000_000)
    ap.add_argument("--spawn-walkers", type=int, default=100_000)
    ap.add_argument("--ntraj-sweep", type=int, default=1, help="0 skips the walker-count sweep")
    ap.add_argument("--served-requests", type=int, default=256)
    ap.add_argument("--served-traj-max", type=float, default=1e6)
    ap.add_argument("--served-arena-gb", type=float, default=48.0)
    ap.add_argument("--served-quantum", type=int, default=400)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
