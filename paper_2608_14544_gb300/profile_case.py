"""The profiling entry point: one solve of a workload through the C ABI
(sample, propagate, reduce), or through the request server with --served, for
ncu; the commands in profiles/ run it.  Prints the wall time; bench.py makes
the measurements.

  python -m paper_2608_14544_gb300.profile_case --config 2 --n-traj 1048576 --steps 160
  python -m paper_2608_14544_gb300.profile_case --config 2 --served --repeat 2
  python -m paper_2608_14544_gb300.profile_case --config lvc4 --modes 64 --n-traj 262144
"""
from __future__ import annotations

import argparse
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="2", help="1-4, or lvc4 (random four-state model)")
    ap.add_argument("--n-traj", type=int, default=None)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--repr", default="adiabatic", choices=["adiabatic", "diabatic"])
    ap.add_argument("--stride", type=int, default=None,
                    help="steps between output times (default: the workload's)")
    ap.add_argument("--spawn", type=int, default=0,
                    help="> 0: a spawning ensemble with this many walker slots per initial walker")
    ap.add_argument("--served", action="store_true",
                    help="submit the solve to the request server (qcl_server_submit / wait)")
    ap.add_argument("--modes", type=int, default=6, help="modes of the lvc4 model")
    ap.add_argument("--modes-in-memory", type=int, default=0, choices=[0, 1, 2],
                    help="QCL_OPT_MODES_IN_MEMORY (0: measured choice, 1: memory, 2: registers)")
    args = ap.parse_args()

    import torch

    from . import build, qcl
    from . import workloads as wl

    build.build()
    torch.cuda.set_device(0)
    qcl.set_option(qcl.OPT_MODES_IN_MEMORY, args.modes_in_memory)
    cfg = wl.lvc4_config(1, args.modes) if args.config == "lvc4" else wl.config(int(args.config))
    cfg["model"]["repr"] = args.repr
    n = args.n_traj or cfg["n_traj"]
    steps = args.steps or cfg["n_steps"]
    stride = args.stride or cfg["out_stride"]
    prec = qcl.PREC_FP32_BULK if args.precision == "fp32" else qcl.PREC_FP64
    if args.served:
        srv = qcl.Server(16 << 30, quantum_steps=steps)
        req = dict(model=cfg["model"], init=cfg["init"], n_traj=n, seed=cfg["seed"],
                   n_steps=steps, dt=cfg["dt"], out_stride=stride)
        for _ in range(args.repeat):
            t0 = time.perf_counter()
            st, obs = srv.wait(srv.submit(req))
            el = time.perf_counter() - t0
            assert st == qcl.REQ_DONE
            print(f"config {args.config} n_traj {n} steps {steps} served: {el * 1e3:.2f} ms, "
                  f"{n * steps / el:.3e} traj-steps/s, trace(t_end) {obs[-1, 32]:.4f}")
        srv.close()
        return
    model = qcl.Model(cfg["model"])
    if args.spawn > 0:
        run = qcl.SpawnRun(model, n, args.spawn * n, cfg["seed"], steps // stride + 1,
                           precision=prec)
    else:
        run = qcl.Run(model, n, cfg["seed"], prec, steps // stride + 1)
    for _ in range(args.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run.sample(cfg["init"])
        run.propagate(steps, cfg["dt"], stride)
        obs = run.observables()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        extra = f", {run.n_live()} walkers at the end" if args.spawn > 0 else ""
        print(f"config {args.config} n_traj {n} steps {steps} {args.precision}: {el * 1e3:.2f} ms, "
              f"{n * steps / el:.3e} traj-steps/s, trace(t_end) {obs[-1, 32]:.4f}{extra}")
    st = run.status()
    assert st["flags"] == 0, st


if __name__ == "__main__":
    main()
