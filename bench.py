"""Benchmark: iterated Jacobi-2D on GB300.

Default workload (one "step" = one full solve): one 8192 x 8192 FP32 grid,
T = 1000 timesteps, interior and boundary uniform[0,1) from seed 0, boundary
fixed.  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the single-grid path has no exchange step); value = all ranks' updates / the
slowest rank's time.

Timing: W untimed steps, then K steps bracketed by a barrier and
cuda.synchronize on both sides, timed with CUDA events on the launching
stream.  The two 256 MiB grids exceed the 126 MB L2, so no L2 flush is needed
between steps.  nvidia-smi clocks are sampled during the timed region.
"""
from __future__ import annotations

import argparse
import glob
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Jacobi-2D GUpdates/s (% HBM roofline); served p50/p99 vs plain launches"
UNIT = "GUpdates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--rows", type=int, default=8192)
    p.add_argument("--cols", type=int, default=8192)
    p.add_argument("--T", type=int, default=1000)
    p.add_argument("--k", type=int, default=0, help="fused depth (0 = library default / autotuned)")
    p.add_argument("--warps", type=int, default=0)
    p.add_argument("--seg-rows", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_name(a):
    return f"jacobi2d_{a.rows}x{a.cols}_f32_T{a.T}"


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """Largest `value` over all ranks (the slowest rank's time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of `world` replicas: all ranks' units / slowest time."""
    return world * units_per_rank / seconds_max


# ------------------------------------------------------------------ clocks ----
CLOCK_FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
                "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(CLOCK_FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) != len(CLOCK_FIELDS):
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- peaks ------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def committed_traffic(kernel_digest: str, workload: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources and workload."""
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path).read()
        m_d = re.search(r"^kernel_digest:\s*(\S+)", text, re.M)
        m_w = re.search(r"^workload:\s*(\S+)", text, re.M)
        m_t = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)", text, re.M)
        if m_d and m_w and m_t and m_d.group(1) == kernel_digest and m_w.group(1) == workload:
            return float(m_t.group(1))
    return None


# ------------------------------------------------------------ CPU oracle -------
def _oracle_step_seconds(g) -> float:
    """Seconds per timestep of the oracle on grid g (setup cost removed)."""
    import oracle
    t0 = time.perf_counter()
    oracle.jacobi2d(g, 1, threads=0)
    t1 = time.perf_counter()
    oracle.jacobi2d(g, 5, threads=0)
    t2 = time.perf_counter()
    return max((t2 - t1) - (t1 - t0), 1e-4) / 4

def cpu_oracle_sample(a, target_s: float):
    """Time the FP64 oracle on a bounded sample of the workload (same grid,
    fewer timesteps, all host threads)."""
    import numpy as np

    import oracle
    from paper_1902_10345_gb300 import inputs

    g = inputs.uniform_grid(a.rows, a.cols, seed=0).astype(np.float32).astype(np.float64)
    threads = oracle.num_threads(0)
    dt = _oracle_step_seconds(g)
    T_s = int(max(2, min(a.T, target_s / dt)))
    t0 = time.perf_counter()
    oracle.jacobi2d(g, T_s, threads=0)
    el = time.perf_counter() - t0
    upd = (a.rows - 2) * (a.cols - 2) * T_s
    return {"value": upd / el / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{a.rows}x{a.cols} grid, FP64 oracle, {T_s} of {a.T} timesteps, {threads} host threads, "
                      f"{el:.1f} s"}


# -------------------------------------------------------------- reference ------
def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1902_10345_gb300 import inputs

    oracle.build()
    g = inputs.uniform_grid(a.rows, a.cols, seed=0).astype(np.float32).astype(np.float64)
    threads = oracle.num_threads(0)
    dt = _oracle_step_seconds(g)
    budget = 150.0 / max(1, a.steps + a.warmup)       # whole run within a few minutes
    T_s = int(max(1, min(a.T, budget / dt)))
    for _ in range(a.warmup):
        oracle.jacobi2d(g, T_s, threads=0)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.jacobi2d(g, T_s, threads=0)
        times.append(time.perf_counter() - t0)
    el = sum(times)
    upd = (a.rows - 2) * (a.cols - 2) * T_s * a.steps
    v = upd / el / 1e9
    sample = f"{a.rows}x{a.cols} grid, FP64 oracle, {T_s} of {a.T} timesteps per step, {threads} host threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1000 * el / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "rows": a.rows, "cols": a.cols, "T": a.T, "sample_T": T_s},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }))


# ------------------------------------------------------------------- ours -------
def run_ours(a):
    import numpy as np
    import torch

    from paper_1902_10345_gb300 import binding, build, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    build.build()
    binding.lib()
    R, C, T = a.rows, a.cols, a.T
    g = inputs.uniform_grid(R, C, seed=0)
    x = torch.from_numpy(g).float().cuda()
    y = torch.empty_like(x)
    cfg = binding.config(kernel=binding.SDFG_KERNEL_AUTO, k=a.k, seg_rows=a.seg_rows, warps=a.warps)
    stream = torch.cuda.current_stream()
    updates = (R - 2) * (C - 2) * T

    for _ in range(max(3, a.warmup)):
        binding.jacobi2d(x, y, T, cfg)
    torch.cuda.synchronize()
    binding.check(binding.sdfg_device_error(True))

    binding.sdfg_stats_reset()
    binding.sdfg_stats_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(a.steps):
            binding.jacobi2d(x, y, T, cfg)
        e1.record(stream)
        barrier()
    binding.sdfg_stats_enable(False)
    ms = e0.elapsed_time(e1)
    launches = {}
    for fam in ("naive", "temporal", "persistent", "reduce", "copy"):
        launches[fam] = binding.sdfg_stats_get(fam)
    binding.sdfg_stats_reset()
    binding.check(binding.sdfg_device_error(True))

    t_max = max_over_ranks(ms, dist, "cuda")
    value = aggregate_rate(updates * a.steps, world, t_max / 1e3) / 1e9

    # end to end through the C ABI with host buffers (pinned), copies timed
    hx = x.cpu().pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    binding.check(binding.sdfg_jacobi2d_host(hx.data_ptr(), hy.data_ptr(), R, C, T, binding.SDFG_F32,
                                             stream.cuda_stream))
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        binding.check(binding.sdfg_jacobi2d_host(hx.data_ptr(), hy.data_ptr(), R, C, T, binding.SDFG_F32,
                                                 stream.cuda_stream))
    e2e_s = time.perf_counter() - t0
    e2e_max = max_over_ranks(e2e_s, dist, "cuda")
    e2e_value = aggregate_rate(updates * a.steps, world, e2e_max) / 1e9
    assert torch.equal(hy.cuda(), y), "end-to-end result differs from the device-resident result"

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (temporal pass): algorithmic bytes per
    # launch = interior points x 2 x 4 B (one read + one write per pass)
    n_tp, ms_tp = launches["temporal"]
    hbm, hbm_src = measured_peaks()
    bytes_per_launch = (R - 2) * (C - 2) * 2 * 4
    achieved = bytes_per_launch / (ms_tp / n_tp / 1e3) / 1e9 if n_tp else None
    from paper_1902_10345_gb300 import build as _b
    digest = _b._digest()[:16]
    traffic = committed_traffic(digest, workload_name(a))
    k_used = a.k or 8
    n_pass = n_tp // a.steps if n_tp else 0
    gpu_launches = sum(v[0] for v in launches.values())
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
            "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else hbm_src,
            "kernel": "temporal_pass_kernel", "k": k_used, "passes_per_step": n_pass,
            "avg_launch_ms": (ms_tp / n_tp) if n_tp else None,
            "roofline_gupdates": hbm * k_used / (2 * 4),
            "kernel_share_of_step": (ms_tp / ms) if ms else None}
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        cpu = cpu_oracle_sample(a, a.cpu_seconds)
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": max(3, a.warmup),
        "ms_per_step": t_max / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(a), "rows": R, "cols": C, "T": T, "k": k_used,
                   "l2": "inputs larger than L2 (two 256 MiB grids), no flush", "parallelism": f"replicas{world}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": R * C * 4, "d2h_bytes_per_step": R * C * 4},
        "clocks": clk.summary(),
        "gpu_launches": gpu_launches,
    }))
    if dist is not None:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
