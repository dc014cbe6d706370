"""Host-side logic of bench.py, without a GPU: the algorithmic flop count of the
roofline, the staleness check of the committed ncu figures, and the reference
arm (the FP64 oracle on the host cores) with its JSON line."""
import json
import os
import subprocess
import sys

import pytest

import bench
from paper_2608_14544_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_flops_per_walker_step_follow_the_per_mode_count():
    # spin-boson form: 10 flops per mode (drift, collective sum, merged kick of
    # two FMA, coupling sum) plus 26 scalar flops; the general form adds the
    # second collective sum (12 per mode)
    assert bench.flops_per_traj_step(wl.config(2)["model"]) == 10 * 3 + 26
    assert bench.flops_per_traj_step(wl.config(4)["model"]) == 10 * 100 + 26
    assert bench.flops_per_traj_step(wl.config(3)["model"]) == 12 * 3 + 26
    assert bench.flops_per_traj_step(wl.random_lvc2(5, seed=1)) == 12 * 5 + 26
    # more than two states: the scope's four-state figure
    assert bench.flops_per_traj_step(wl.random_lvc4(3)) == bench.FLOPS_NSTATE


def test_profiled_figures_are_dropped_when_the_sources_change(tmp_path):
    srcs = [tmp_path / "a.cu", tmp_path / "b.cuh"]
    srcs[0].write_text("kernel one\n")
    srcs[1].write_text("header\n")
    paths = [str(p) for p in srcs]
    h = bench.kernel_source_hash(paths)
    summary = tmp_path / "k.md"
    summary.write_text("# k\n\ninstructions_per_walker_step: 91.4\n"
                       "traffic_bytes_per_launch: 664770507\n"
                       f"traffic_source_sha256_prefix: {h}\n")
    assert bench._profiled(paths, str(summary), "instructions_per_walker_step") == 91.4
    assert bench._profiled_traffic(paths, str(summary)) == 664770507.0
    assert bench._profiled(paths, str(summary), "missing_key") is None
    # the order of the sources is part of the hash
    assert bench._profiled(paths[::-1], str(summary), "instructions_per_walker_step") is None
    srcs[1].write_text("header, changed\n")
    assert bench._profiled_traffic(paths, str(summary)) is None
    assert bench._profiled_traffic(paths, str(tmp_path / "absent.md")) is None


def test_committed_headline_summary_carries_the_figures():
    txt = open(os.path.join(ROOT, "profiles", "k_bulk2_sb3mode.md")).read()
    vals = dict(ln.split(":", 1) for ln in txt.splitlines()
                if ln.startswith(("instructions_per_walker_step:", "traffic_bytes_per_launch:",
                                  "traffic_source_sha256_prefix:")))
    assert float(vals["instructions_per_walker_step"]) > 0
    assert float(vals["traffic_bytes_per_launch"]) > 0
    assert len(vals["traffic_source_sha256_prefix"].strip()) == 16


def test_issue_slot_roofline_arithmetic():
    r = bench._issue_roofline(2.0e11, 152, 2070.0)
    if r is None:  # the committed summary is stale for the current sources
        pytest.skip("no current instruction count")
    ipw = r["instructions_per_walker_step"]
    assert r["achieved_warp_instr_per_s"] == pytest.approx(2.0e11 * ipw / 32)
    assert r["peak_warp_instr_per_s"] == pytest.approx(152 * 4 * 2070e6)
    assert r["frac"] == pytest.approx(r["achieved_warp_instr_per_s"] / r["peak_warp_instr_per_s"])


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "traj-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "traj-steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the same metric and configuration as the GPU arm's line
    assert d["config"] == bench.bench_config(wl.config(bench.WORKLOAD), 1)
