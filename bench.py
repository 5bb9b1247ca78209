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
import math
import os
import re
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Jacobi-2D GUpdates/s (% HBM roofline); served p50/p99 vs plain launches"
UNIT = "GUpdates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--rows", type=int, default=8192)
    p.add_argument("--cols", type=int, default=8192)
    p.add_argument("--T", type=int, default=1000)
    p.add_argument("--k", type=int, default=0, help="fused depth (0 = library default / autotuned)")
    p.add_argument("--warps", type=int, default=0)
    p.add_argument("--seg-rows", type=int, default=0)
    p.add_argument("--kernel", choices=["persistent", "temporal", "resident", "skewed"], default="skewed")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--workload", choices=["single", "batch", "precision", "serve", "paper", "3d", "sor"],
                   default="single",
                   help="single: 8192^2 FP32 T=1000 (the default line); batch: 512 uneven grids in one "
                        "persistent launch; precision: 4 x 16384^2 T=500 FP32 and BF16; serve: Laplace requests; "
                        "3d: the 7-point stencil on a 512^3 FP32 box, T=100; sor: red-black SOR on the 8192^2 "
                        "FP32 grid, omega 1.9, 1000 iterations")
    p.add_argument("--omega", type=float, default=1.9, help="sor: relaxation factor")
    p.add_argument("--size3d", type=int, default=512, help="3d: box edge")
    p.add_argument("--T3d", type=int, default=100, help="3d: timesteps")
    p.add_argument("--requests", type=int, default=2000, help="serve: number of requests")
    p.add_argument("--rho", type=float, default=0.9, help="serve: arrival rate as a fraction of served capacity")
    p.add_argument("--plain-seconds", type=float, default=120.0,
                   help="serve: wall-time cap of the plain-launch replay (a prefix of the trace)")
    p.add_argument("--precision-grids", type=int, default=4, help="precision: 16384^2 grids per storage type")
    p.add_argument("--batch-grids", type=int, default=512,
                   help="batch: grids in the batch (the first n of the seeded 512; smaller batches for profiling)")
    p.add_argument("--line-requests", type=int, default=1000,
                   help="default line: served requests (a prefix of the seeded 10,000-request trace)")
    p.add_argument("--line-plain-seconds", type=float, default=90.0,
                   help="default line: wall-time cap of the plain-launch replay")
    p.add_argument("--no-extra-blocks", action="store_true",
                   help="default line: skip the served, batch and precision blocks")
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
        self.path = os.path.join(tempfile.gettempdir(), f"sdfg_bench_clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(CLOCK_FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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


def fp32_lane_ops_per_update(family: str, k: int, seg_rows: int, warp_cols: int = 128):
    """FP32-pipe lane-ops per useful update of the reassociated pipe at depth
    k, and the redundant-work factor of the kernel's tiles.  Per lane and 4
    columns a fused level issues 5 packed FP32x2 adds (2 lane-ops each) and 4
    scalar adds: 14 lane-ops, 3.5 per update; the pass's 0.2^k scale is one
    FFMA2 + one FMUL2 per 4 columns (1 lane-op per point per pass, 1/k per
    update).  Strips compute warp_cols columns for warp_cols - 2h stored
    (h = k rounded up to 4 columns); the persistent and per-pass kernels
    recompute 2k rows per segment of seg_rows rows, the chain kernel 2k rows
    per chain of seg_rows rows."""
    h = -(-max(k, 1) // 4) * 4
    cols = warp_cols / (warp_cols - 2 * h)
    rows = (seg_rows + 2 * k) / seg_rows if family in ("persistent", "temporal", "skewed") and seg_rows else 1.0
    return 3.5 + 1.0 / k, cols * rows


def kernel_code(binding, name: str) -> int:
    """The library's kernel-family code for a --kernel name."""
    return {"persistent": binding.SDFG_KERNEL_PERSISTENT, "temporal": binding.SDFG_KERNEL_TEMPORAL,
            "resident": binding.SDFG_KERNEL_RESIDENT, "skewed": binding.SDFG_KERNEL_SKEWED}[name]


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

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_sample(a, target_s: float):
    """Time the FP64 oracle on a bounded sample of the workload (same grid,
    fewer timesteps): on all host threads, and on one thread for a quarter of
    the time."""
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
    # single thread: a few timesteps, about target_s / 4 of wall time (one
    # thread takes at most `threads` times the measured all-thread step time)
    T_1 = int(max(1, min(a.T, 0.25 * target_s / (el / T_s * threads))))
    t0 = time.perf_counter()
    oracle.jacobi2d(g, T_1, threads=1)
    el1 = time.perf_counter() - t0
    return {"value": upd / el / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{a.rows}x{a.cols} grid, FP64 oracle, {T_s} of {a.T} timesteps, {threads} host threads, "
                      f"{el:.1f} s",
            "cpu_model": cpu_model(),
            "single_thread": {"value": (a.rows - 2) * (a.cols - 2) * T_1 / el1 / 1e9, "unit": UNIT, "cores": 1,
                              "sample": f"{T_1} of {a.T} timesteps, 1 thread, {el1:.1f} s"}}


def median_ci95(xs):
    """Median of xs and a distribution-free 95% confidence interval for it
    (order statistics at n/2 -+ 1.96 sqrt(n)/2)."""
    v = sorted(xs)
    n = len(v)
    if n == 0:
        return None, [None, None]
    med = v[n // 2] if n % 2 else 0.5 * (v[n // 2 - 1] + v[n // 2])
    half = 1.96 * math.sqrt(n) / 2
    lo = max(0, int(math.floor(n / 2 - half)) - 1)
    hi = min(n - 1, int(math.ceil(n / 2 + half)) - 1)
    return med, [v[lo], v[hi]]


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
    # the launch configuration timed here (and used by the full-size parity test)
    cfg = binding.config(kernel=kernel_code(binding, a.kernel), k=a.k or 8,
                         seg_rows=a.seg_rows or (640 if a.kernel == "skewed" else 128), warps=a.warps or 4)
    stream = torch.cuda.current_stream()
    updates = (R - 2) * (C - 2) * T

    for _ in range(max(3, a.warmup)):
        binding.jacobi2d(x, y, T, cfg)
    torch.cuda.synchronize()
    binding.check(binding.sdfg_device_error(True))

    binding.sdfg_stats_reset()
    binding.sdfg_stats_enable(True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    with ClockSampler(local) as clk:
        barrier()
        evs[0].record(stream)
        for i in range(a.steps):
            binding.jacobi2d(x, y, T, cfg)
            evs[i + 1].record(stream)
        barrier()
    binding.sdfg_stats_enable(False)
    ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(a.steps)]
    med_ms, ci_ms = median_ci95(step_ms)
    launches = {}
    for fam in ("naive", "temporal", "persistent", "reduce", "copy", "stencil3d", "sor", "resident", "skewed"):
        launches[fam] = binding.sdfg_stats_get(fam)
    binding.sdfg_stats_reset()
    binding.check(binding.sdfg_device_error(True))

    t_max = max_over_ranks(ms, dist, "cuda")
    value = aggregate_rate(updates * a.steps, world, t_max / 1e3) / 1e9

    # end to end through the C ABI with host buffers (pinned), copies timed;
    # the library times its own host <-> device copies (stats families h2d, d2h).
    # Serial: one sdfg_jacobi2d_host call per step (copy in, solve, copy out,
    # wait).  Pipelined (the e2e value): the K steps as K independent solves
    # in one sdfg_jacobi2d_host_many call, each still copying its own input in
    # and its result out, the copies of one overlapping the next one's solve;
    # two pairs of host buffers alternate, so no two solves in flight share one.
    hx = x.cpu().pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    hx2 = hx.clone().pin_memory()
    hy2 = torch.empty_like(hx).pin_memory()
    binding.check(binding.sdfg_jacobi2d_host(hx.data_ptr(), hy.data_ptr(), R, C, T, binding.SDFG_F32,
                                             stream.cuda_stream))
    barrier()
    binding.sdfg_stats_reset()
    binding.sdfg_stats_enable(True)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        binding.check(binding.sdfg_jacobi2d_host(hx.data_ptr(), hy.data_ptr(), R, C, T, binding.SDFG_F32,
                                                 stream.cuda_stream))
    e2e_serial_s = time.perf_counter() - t0
    binding.sdfg_stats_enable(False)
    e2e_launches = {f: binding.sdfg_stats_get(f) for f in ("h2d", "d2h", "skewed", "persistent", "copy")}
    binding.sdfg_stats_reset()
    ins = [hx.data_ptr(), hx2.data_ptr()]
    outs = [hy.data_ptr(), hy2.data_ptr()]
    binding.check(binding.sdfg_jacobi2d_host_many(ins, outs, R, C, T, binding.SDFG_F32, stream.cuda_stream))
    barrier()
    t0 = time.perf_counter()
    binding.check(binding.sdfg_jacobi2d_host_many([ins[i & 1] for i in range(a.steps)],
                                                  [outs[i & 1] for i in range(a.steps)], R, C, T,
                                                  binding.SDFG_F32, stream.cuda_stream))
    e2e_s = time.perf_counter() - t0
    # the same call again, untimed, with the library's per-copy event timing
    # on: how many copies each solve made, and how long they took
    binding.sdfg_stats_reset()
    binding.sdfg_stats_enable(True)
    t0 = time.perf_counter()
    binding.check(binding.sdfg_jacobi2d_host_many([ins[i & 1] for i in range(a.steps)],
                                                  [outs[i & 1] for i in range(a.steps)], R, C, T,
                                                  binding.SDFG_F32, stream.cuda_stream))
    e2e_stats_s = time.perf_counter() - t0
    binding.sdfg_stats_enable(False)
    pipe_copies = {f: binding.sdfg_stats_get(f) for f in ("h2d", "d2h")}
    binding.sdfg_stats_reset()
    e2e_serial_max = max_over_ranks(e2e_serial_s, dist, "cuda")
    e2e_serial_value = aggregate_rate(updates * a.steps, world, e2e_serial_max) / 1e9
    e2e_max = max_over_ranks(e2e_s, dist, "cuda")
    e2e_value = aggregate_rate(updates * a.steps, world, e2e_max) / 1e9
    # the host entry point runs the library's default for this shape (the
    # chain kernel, k = 8, 640-row chains); FP32 results depend only on the
    # kernel's geometry (which units reassociate the sum, and how), so they
    # are bitwise equal to the device-resident run in that geometry and agree
    # to the FP32 parity tolerance otherwise
    for h in (hy, hy2):
        if a.kernel == "skewed" and (cfg.k, cfg.seg_rows) == (8, 640):
            assert torch.equal(h.cuda(), y), "end-to-end result differs from the device-resident result"
        else:
            assert (h.cuda() - y).abs().max().item() <= 1e-4, "end-to-end result differs from the device-resident result"
    h2d_ms = e2e_launches["h2d"][1] / a.steps
    d2h_ms = e2e_launches["d2h"][1] / a.steps
    copy_ms = h2d_ms + d2h_ms
    e2e_kernel_ms = sum(e2e_launches[f][1] for f in ("skewed", "persistent", "copy")) / a.steps

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel: algorithmic bytes = interior points x
    # 2 x 4 B per pass (one read + one write per pass of k fused steps)
    fam = max(("temporal", "persistent", "resident", "skewed"), key=lambda f: launches[f][1])
    n_tp, ms_tp = launches[fam]
    hbm, hbm_src = measured_peaks()
    k_used = cfg.k
    passes_per_step = -(-T // k_used)
    bytes_per_launch = (R - 2) * (C - 2) * 2 * 4 * (passes_per_step if fam in ("persistent", "skewed") else 1)
    achieved = bytes_per_launch / (ms_tp / n_tp / 1e3) / 1e9 if n_tp else None
    # FP32-pipe ceiling: 152 SMs x 128 FP32 lanes at the max SM clock; the
    # lane-ops the reassociated pipe issues per useful update, times the
    # redundancy of its tiles
    alu_peak = 152 * 128 * 2.07e9 / 1e12
    ops_per_update, redundancy = fp32_lane_ops_per_update(fam, k_used, cfg.seg_rows)
    alu_achieved = ops_per_update * redundancy * value / 1e3
    from paper_1902_10345_gb300 import build as _b
    digest = _b.kernel_digest(_b.KERNEL_FILES_CHAIN if fam == "skewed" else None)
    traffic = committed_traffic(digest, workload_name(a))
    gpu_launches = sum(v[0] for v in launches.values())
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
            "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else hbm_src,
            "kernel": f"{fam}_kernel", "k": k_used, "passes_per_step": passes_per_step,
            "launches_per_step": n_tp / a.steps if n_tp else 0,
            "avg_launch_ms": (ms_tp / n_tp) if n_tp else None,
            "roofline_gupdates": hbm * k_used / (2 * 4),
            "kernel_share_of_step": (ms_tp / ms) if ms else None,
            "secondary": {"bound": "alu", "unit": "T FP32 lane-ops/s", "achieved": alu_achieved, "peak": alu_peak,
                          "frac": alu_achieved / alu_peak, "lane_ops_per_update": ops_per_update,
                          "tile_redundancy": redundancy,
                          "ceiling_gupdates": 1e3 * alu_peak / (ops_per_update * redundancy),
                          "note": "FP32-pipe lane-ops the reassociated pipe issues per update (3.5 adds + the "
                                  "once-per-pass 0.2^k scale), times the overlapped tiles' redundant work, vs "
                                  "152 SMs x 128 FP32 lanes x 2.07 GHz"}}
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        cpu = cpu_oracle_sample(a, a.cpu_seconds)
    # the rest of the metric and of the workload set, on one GPU: served
    # p50/p99 against plain launches, the 512-grid batch, and the precision
    # sweep's errors on every element (replicas at N > 1 run the line alone)
    extra = {}
    if world == 1 and not a.no_extra_blocks:
        for key, fn in (("served", lambda: measure_serve(a, a.line_requests, a.rho, a.line_plain_seconds)),
                        ("batch", lambda: measure_batch(a, 10, 3)),
                        ("precision", lambda: measure_precision(a, a.precision_grids))):
            t0 = time.perf_counter()
            extra[key] = fn()
            extra[key]["wall_s"] = time.perf_counter() - t0
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": max(3, a.warmup),
        "ms_per_step": t_max / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "step_ms": {"median": med_ms, "ci95": ci_ms, "min": min(step_ms), "max": max(step_ms),
                    "median_gupdates": updates / (med_ms / 1e3) / 1e9 if med_ms else None},
        "config": {"workload": workload_name(a), "rows": R, "cols": C, "T": T, "k": k_used,
                   "kernel": a.kernel, "seg_rows": cfg.seg_rows, "warps_per_cta": cfg.warps,
                   "l2": "inputs larger than L2 (two 256 MiB grids), no flush", "parallelism": f"replicas{world}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": R * C * 4, "d2h_bytes_per_step": R * C * 4,
                "ms_per_step": 1e3 * e2e_max / a.steps,
                "api": "sdfg_jacobi2d_host_many: the K steps as K independent host-to-host solves, "
                       "each copying its input in and its result out, pipelined on two device slots",
                "h2d_copies": pipe_copies["h2d"][0], "d2h_copies": pipe_copies["d2h"][0],
                "copy_ms_per_step": (pipe_copies["h2d"][1] + pipe_copies["d2h"][1]) / a.steps,
                "ms_per_step_with_copy_timing": 1e3 * e2e_stats_s / a.steps,
                "note": "copies counted and timed (CUDA events per copy) in a second, untimed call of the same "
                        "K solves; copy_ms_per_step is each solve's two copies, overlapped with the other "
                        "slot's solve",
                "serial": {"value": e2e_serial_value, "unit": UNIT, "ms_per_step": 1e3 * e2e_serial_max / a.steps,
                           "api": "sdfg_jacobi2d_host, one call per step",
                           "copy_ms_per_step": copy_ms, "h2d_ms_per_step": h2d_ms, "d2h_ms_per_step": d2h_ms,
                           "kernel_ms_per_step": e2e_kernel_ms,
                           "copy_gbs": 2 * R * C * 4 / (copy_ms / 1e3) / 1e9 if copy_ms else None,
                           "note": "copy and kernel times are the library's own CUDA-event timings inside "
                                   "sdfg_jacobi2d_host; ms_per_step - copy - kernel is host-side overhead"}},
        "clocks": clk.summary(),
        "gpu_launches": gpu_launches,
        **extra,
    }))
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------- batch -------
def _padded(R, C, dtype, device="cuda"):
    import torch
    ld = (C + 3) // 4 * 4
    return torch.zeros((R, ld), dtype=dtype, device=device)[:, :C]


def measure_batch(a, steps: int, warmup: int, n_grids: int = 512):
    """512 uneven grids (rows, cols log-uniform in [64, 2048], T in [50, 500])
    in ONE persistent launch, replayed through a captured CUDA graph; k and
    the segment height from the project's batch autotuner unless --k or
    --seg-rows fix them.  n_grids < 512 takes the first n_grids of the same
    seeded batch (for profiling).  Returns the block of the JSON line."""
    import ctypes

    import torch

    from paper_1902_10345_gb300 import binding, build, inputs

    build.build()
    L = binding.lib()
    specs = inputs.batch_specs(512, seed=0)[:n_grids]
    wl = "jacobi2d_batch512_uneven_f32" if n_grids == 512 else f"jacobi2d_batch{n_grids}of512_uneven_f32"
    xs, ys, descs = [], [], []
    for sp in specs:
        x = _padded(sp.rows, sp.cols, torch.float32)
        x.copy_(torch.from_numpy(inputs.batch_grid(sp)).float())
        y = _padded(sp.rows, sp.cols, torch.float32)
        xs.append(x)
        ys.append(y)
        descs.append(binding.desc_for(x, y, sp.T))
    updates = sum((sp.rows - 2) * (sp.cols - 2) * sp.T for sp in specs)
    if a.k or (a.seg_rows and a.workload == "batch"):
        cfg = binding.config(kernel=kernel_code(binding, a.kernel if a.kernel in ("persistent", "skewed")
                                                else "persistent"),
                             k=a.k or 8, seg_rows=a.seg_rows or 96, warps=a.warps or 4)
        tuned = False
    else:
        # the project's autotuner picks k and the segment height on this batch
        cfg = binding.sdfg_autotune_batch(descs, 64)
        tuned = True
    arr = (binding.sdfg_desc * len(descs))(*descs)
    plan = ctypes.c_void_p()
    stream = torch.cuda.current_stream()
    binding.check(L.sdfg_batch_plan_create(ctypes.byref(plan), arr, len(descs), 64, ctypes.byref(cfg), 0))
    for _ in range(max(3, warmup)):
        binding.check(L.sdfg_batch_plan_run(plan, stream.cuda_stream))
    binding.check(L.sdfg_batch_plan_results(plan, arr, len(descs)))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            binding.check(L.sdfg_batch_plan_run(plan, stream.cuda_stream))
        e1.record(stream)
        torch.cuda.synchronize()
    binding.check(L.sdfg_batch_plan_results(plan, arr, len(descs)))
    ms = e0.elapsed_time(e1)
    binding.check(L.sdfg_batch_plan_destroy(plan))
    assert all(d.status == 0 and d.steps_done == sp.T for d, sp in zip(arr, specs))
    value = updates * steps / (ms / 1e3) / 1e9
    k = cfg.k
    # passes of the plan: plan_passes(T, k) = T // k passes of k, then the remainder in powers of two
    def n_passes(T):
        return T // k + bin(T % k).count("1")
    passes = sum(n_passes(sp.T) for sp in specs)
    bytes_per_step = sum((sp.rows - 2) * (sp.cols - 2) * 2 * 4 * n_passes(sp.T) for sp in specs)
    hbm, src = measured_peaks()
    achieved = bytes_per_step / (ms / steps / 1e3) / 1e9
    persistent = cfg.kernel != binding.SDFG_KERNEL_SKEWED
    traffic = committed_traffic(build.kernel_digest(None), wl) if persistent else None
    # kernels one replay launches (no grid of this batch solves to a tolerance,
    # so no finalize launch): the persistent kernel; or the ring copy and the
    # chain kernel, plus the persistent kernel for grids under 2^20 points
    if persistent:
        per_step = 1
    else:
        per_step = 2 + (1 if any(sp.rows * sp.cols < (1 << 20) for sp in specs) else 0)
    del xs, ys
    torch.cuda.empty_cache()
    return {
        "value": value, "unit": UNIT, "steps": steps, "warmup": max(3, warmup), "ms_per_step": ms / steps,
        "launches_per_step": per_step,
        "config": {"workload": wl, "grids": n_grids, "updates_per_step": updates,
                   "k": k, "seg_rows": cfg.seg_rows, "autotuned": tuned, "passes_per_step": passes,
                   "kernel": ("chain kernel" if cfg.kernel == binding.SDFG_KERNEL_SKEWED else "persistent kernel")
                             + " (one launch per step, replayed from a captured CUDA graph)",
                   "layout": "each grid pitched to a multiple of 4 columns (16-byte rows)",
                   "l2": "1.3 GB resident, larger than L2, no flush" if n_grids == 512 else "first grids of the batch"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "peak_source": src, "roofline_gupdates": hbm * k / 8,
                     "note": "algorithmic bytes 2 x 4 B per interior point and pass of k steps; whole step timed"},
        "clocks": clk.summary(),
    }


def run_batch(a):
    b = measure_batch(a, a.steps, a.warmup, a.batch_grids)
    print(json.dumps({"metric": METRIC, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                      "gpu_launches": b["launches_per_step"] * a.steps, **b}))


# --------------------------------------------------------------- precision -------
def measure_precision(a, grids: int = 4):
    """`grids` grids of 16384^2 (the sinusoid field), T = 500, with FP32
    storage and with BF16 storage (FP32 arithmetic): throughput of each, and
    each result's max-abs and RMS error against the FP64 oracle on EVERY
    element.  The oracle starts from exactly the values the GPU received (the
    field rounded to the storage type) and runs on all host threads; the
    input's own rounding error is reported beside it."""
    import numpy as np
    import torch

    import oracle
    from paper_1902_10345_gb300 import binding, build, inputs

    build.build()
    binding.lib()
    oracle.build()
    n, T = 16384, 500
    out = {}
    stream = torch.cuda.current_stream()
    oracle_s = 0.0
    for dt_name, tdt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        ms_total, max_err, sq, cnt, q_err = 0.0, 0.0, 0.0, 0, 0.0
        for seed in range(grids):
            f64 = inputs.sinusoid_field_device(n, seed=seed)
            x = f64.to(tdt)
            q_err = max(q_err, float((x.double() - f64).abs().max()))
            del f64
            y = torch.empty_like(x)
            binding.jacobi2d(x, y, T)                       # warm-up / plan
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            binding.jacobi2d(x, y, T)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_total += e0.elapsed_time(e1)
            xh = x.double().cpu().numpy()
            t0 = time.perf_counter()
            want = oracle.jacobi2d(xh, T, threads=0)
            oracle_s += time.perf_counter() - t0
            del xh
            d = y.double().cpu().numpy()
            d -= want
            del want
            max_err = max(max_err, float(np.abs(d).max()))
            sq += float(np.einsum("ij,ij->", d, d))
            cnt += d.size
            del d, x, y
            torch.cuda.empty_cache()
        updates = grids * (n - 2) * (n - 2) * T
        out[dt_name] = {"gupdates_per_s": updates / (ms_total / 1e3) / 1e9, "ms": ms_total,
                        "max_abs_err": max_err, "rms_err": (sq / cnt) ** 0.5,
                        "input_quantisation_max_abs": q_err,
                        "compared": f"every element of {grids} grids of {n}x{n} (FP64 oracle, all host threads)"}
    return {"workload": f"precision_{grids}x{n}sq_T{T}_sinusoid", "results": out,
            "tolerance": {"f32": 1e-4, "bf16": 2e-2}, "oracle_seconds": oracle_s,
            "kernel": "library default for the shape (chain kernel, k = 8)"}


def run_precision(a):
    print(json.dumps({"metric": METRIC, "unit": UNIT, **measure_precision(a, a.precision_grids)}))


# ------------------------------------------------------------------- paper -------
def run_paper(a):
    """The paper's Jacobi workload (Sec. 6.1): 2048^2, T = 1024, FP32, constant
    (zero) boundary; interior uniform[0,1) from seed 0.  The grid (2 x 16 MiB)
    lives in L2, so this is a compute-bound case; k and the kernel are chosen
    by the autotuner."""
    import torch

    from paper_1902_10345_gb300 import binding, build, inputs

    build.build()
    binding.lib()
    R = C = 2048
    T = 1024
    g = inputs.uniform_grid(R, C, seed=0)
    g[0, :] = g[-1, :] = 0.0
    g[:, 0] = g[:, -1] = 0.0
    x = torch.from_numpy(g).float().cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    if a.k or a.seg_rows:
        cfg = binding.config(kernel=kernel_code(binding, a.kernel), k=a.k or 8, seg_rows=a.seg_rows,
                             warps=a.warps or 4)
    else:
        cfg = binding.sdfg_autotune(R, C, T, binding.SDFG_F32, stream.cuda_stream)
    for _ in range(max(3, a.warmup)):
        binding.jacobi2d(x, y, T, cfg)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        binding.jacobi2d(x, y, T, cfg)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    print(json.dumps({"metric": METRIC, "unit": UNIT, "workload": "paper_jacobi_2048sq_T1024_f32_zero_boundary",
                      "value": (R - 2) * (C - 2) * T / (ms / 1e3) / 1e9, "ms_per_solve": ms,
                      "config": {"kernel": cfg.kernel, "k": cfg.k, "seg_rows": cfg.seg_rows, "warps": cfg.warps},
                      "note": "paper's own figure for this workload is in a lost plot (P100); context only"}))


# ---------------------------------------------------------------------- 3-D -------
def run_3d(a):
    """The 7-point stencil on an n^3 FP32 box (uniform [0,1) from seed 0,
    shell included), T timesteps, one launch per step; inputs (2 x 512 MiB at
    n = 512) are larger than L2."""
    import numpy as np
    import torch

    from paper_1902_10345_gb300 import binding, build, inputs

    build.build()
    binding.lib()
    n, T = a.size3d, a.T3d
    g = inputs.uniform_box(n, n, n, seed=0)
    x = torch.from_numpy(g).float().cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    updates = (n - 2) ** 3 * T
    for _ in range(max(3, a.warmup)):
        binding.jacobi3d(x, y, T)
    torch.cuda.synchronize()
    binding.check(binding.sdfg_device_error(True))
    binding.sdfg_stats_reset()
    binding.sdfg_stats_enable(True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        evs[0].record(stream)
        for i in range(a.steps):
            binding.jacobi3d(x, y, T)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
    binding.sdfg_stats_enable(False)
    ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(a.steps)]
    med_ms, ci_ms = median_ci95(step_ms)
    n_k, ms_k = binding.sdfg_stats_get("stencil3d")
    n_c, _ = binding.sdfg_stats_get("copy")
    binding.sdfg_stats_reset()
    binding.check(binding.sdfg_device_error(True))
    value = updates * a.steps / (ms / 1e3) / 1e9
    # end to end through the public API with host buffers: pinned host ->
    # device, T steps, device -> pinned host, every step
    hx = x.cpu().pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    dx = torch.empty_like(x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        dx.copy_(hx, non_blocking=True)
        binding.jacobi3d(dx, y, T)
        hy.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    assert torch.equal(hy.cuda(), y), "end-to-end result differs from the device-resident result"
    hbm, hbm_src = measured_peaks()
    bytes_per_launch = (n - 2) ** 3 * 2 * 4        # one read and one write per interior point and step
    achieved = bytes_per_launch / (ms_k / n_k / 1e3) / 1e9 if n_k else None
    wl = f"jacobi3d_{n}cube_f32_T{T}"
    traffic = committed_traffic(build.kernel_digest(build.KERNEL_FILES_3D), wl)
    cpu = None
    if not a.no_cpu_baseline:
        import oracle
        oracle.build()
        gd = x.double().cpu().numpy()
        # seconds per step with the setup (allocation, copies) removed
        t0 = time.perf_counter()
        oracle.jacobi3d(gd, 1, threads=0)
        t1 = time.perf_counter()
        oracle.jacobi3d(gd, 3, threads=0)
        t2 = time.perf_counter()
        dt1 = max((t2 - t1) - (t1 - t0), 1e-3) / 2
        T_s = int(max(1, min(T, a.cpu_seconds / dt1)))
        t0 = time.perf_counter()
        oracle.jacobi3d(gd, T_s, threads=0)
        el = time.perf_counter() - t0
        cpu = {"value": (n - 2) ** 3 * T_s / el / 1e9, "unit": UNIT, "cores": oracle.num_threads(0), "kind": "oracle",
               "sample": f"{n}^3 box, FP64 3-D oracle, {T_s} of {T} timesteps, all host threads, {el:.1f} s",
               "cpu_model": cpu_model()}
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": max(3, a.warmup),
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "step_ms": {"median": med_ms, "ci95": ci_ms, "min": min(step_ms), "max": max(step_ms)},
        "config": {"workload": wl, "depth": n, "rows": n, "cols": n, "T": T,
                   "kernel": "stencil3d (one launch per step)", "tile": "16 rows x 120 cols, planes streamed",
                   "l2": f"inputs larger than L2 (two {n ** 3 * 4 >> 20} MiB boxes), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                     "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else hbm_src,
                     "kernel": "jacobi3d_kernel", "k": 1, "launches_per_step": n_k / a.steps if n_k else 0,
                     "avg_launch_ms": (ms_k / n_k) if n_k else None, "roofline_gupdates": hbm / 8,
                     "kernel_share_of_step": (ms_k / ms) if ms else None},
        "cpu_baseline": cpu,
        "e2e": {"value": updates * a.steps / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": n ** 3 * 4,
                "d2h_bytes_per_step": n ** 3 * 4},
        "clocks": clk.summary(),
        "gpu_launches": n_k + n_c,
    }))


# ---------------------------------------------------------------------- SOR -------
def run_sor(a):
    """Red-black SOR on the default grid (8192^2 FP32, uniform [0,1) from
    seed 0, boundary ring fixed), a.T iterations of relaxation a.omega, one
    launch per iteration; inputs (2 x 256 MiB) are larger than L2."""
    import torch

    from paper_1902_10345_gb300 import binding, build, inputs

    build.build()
    binding.lib()
    R, C, T, om = a.rows, a.cols, a.T, a.omega
    x = torch.from_numpy(inputs.uniform_grid(R, C, seed=0)).float().cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    updates = (R - 2) * (C - 2) * T
    for _ in range(max(3, a.warmup)):
        binding.sor2d(x, y, T, om)
    torch.cuda.synchronize()
    binding.check(binding.sdfg_device_error(True))
    binding.sdfg_stats_reset()
    binding.sdfg_stats_enable(True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        evs[0].record(stream)
        for i in range(a.steps):
            binding.sor2d(x, y, T, om)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
    binding.sdfg_stats_enable(False)
    ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(a.steps)]
    med_ms, ci_ms = median_ci95(step_ms)
    n_k, ms_k = binding.sdfg_stats_get("sor")
    n_c, _ = binding.sdfg_stats_get("copy")
    binding.sdfg_stats_reset()
    binding.check(binding.sdfg_device_error(True))
    value = updates * a.steps / (ms / 1e3) / 1e9
    hx = x.cpu().pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    dx = torch.empty_like(x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        dx.copy_(hx, non_blocking=True)
        binding.sor2d(dx, y, T, om)
        hy.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    assert torch.equal(hy.cuda(), y), "end-to-end result differs from the device-resident result"
    hbm, hbm_src = measured_peaks()
    iters_per_launch = 4                              # FP32: four red-black iterations per launch
    bytes_per_launch = (R - 2) * (C - 2) * 2 * 4     # one read and one write per interior point and launch
    achieved = bytes_per_launch / (ms_k / n_k / 1e3) / 1e9 if n_k else None
    wl = f"sor2d_{R}x{C}_f32_T{T}_omega{om:g}"
    traffic = committed_traffic(build.kernel_digest(build.KERNEL_FILES_SOR), wl)
    cpu = None
    if not a.no_cpu_baseline:
        import oracle
        oracle.build()
        gd = x.double().cpu().numpy()
        t0 = time.perf_counter()
        oracle.sor2d(gd, 1, om)
        t1 = time.perf_counter()
        oracle.sor2d(gd, 3, om)
        t2 = time.perf_counter()
        dt1 = max((t2 - t1) - (t1 - t0), 1e-3) / 2
        T_s = int(max(1, min(T, a.cpu_seconds / dt1)))
        t0 = time.perf_counter()
        oracle.sor2d(gd, T_s, om)
        el = time.perf_counter() - t0
        cpu = {"value": (R - 2) * (C - 2) * T_s / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{R}x{C} grid, FP64 red-black SOR oracle (one thread), {T_s} of {T} iterations, {el:.1f} s",
               "cpu_model": cpu_model()}
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": max(3, a.warmup),
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "step_ms": {"median": med_ms, "ci95": ci_ms, "min": min(step_ms), "max": max(step_ms)},
        "config": {"workload": wl, "rows": R, "cols": C, "T": T, "omega": om,
                   "kernel": "sor2d (4 red-black iterations per launch)", "tile": "64 rows x 112 cols (10 rows per warp in registers), 4 iterations per launch",
                   "l2": "inputs larger than L2 (two 256 MiB grids), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                     "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else hbm_src,
                     "kernel": "sor2d_reg_kernel", "k": iters_per_launch,
                     "launches_per_step": n_k / a.steps if n_k else 0,
                     "avg_launch_ms": (ms_k / n_k) if n_k else None,
                     "roofline_gupdates": hbm * iters_per_launch / 8,
                     "kernel_share_of_step": (ms_k / ms) if ms else None},
        "cpu_baseline": cpu,
        "e2e": {"value": updates * a.steps / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": R * C * 4,
                "d2h_bytes_per_step": R * C * 4},
        "clocks": clk.summary(),
        "gpu_launches": n_k + n_c,
    }))


# ------------------------------------------------------------------- serve -------
def _pct(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def measure_serve(a, n: int, rho: float, plain_seconds: float):
    """Served Laplace solves: the first n requests of the seeded served
    trace (sides log-uniform in [32, 4096], boundary x^2 - y^2 + noise, zero
    interior, FP32, relative residual 1e-6 or 20000 steps), 40 GB budget.
    Capacity first (all requests at t = 0), then a Poisson arrival trace at
    rho x capacity replayed against (1) the continuous-batching server and
    (2) plain launches: one blocking sdfg_jacobi2d_solve per request in
    arrival order, in the server's geometry (same fused depth and segment
    height), so both stop every request at the same step: equal accuracy."""
    import ctypes
    import threading

    import numpy as np
    import torch

    from paper_1902_10345_gb300 import binding, build, inputs

    build.build()
    L = binding.lib()
    reqs = inputs.served_requests(n, seed=0)
    xs = [inputs.laplace_request_grid_device(r, dtype=torch.float32) for r in reqs]
    ys = [torch.zeros_like(x) for x in xs]
    tol, cap, stride, quantum = 1e-6, 20000, 64, 256
    budget = 40 << 30
    # the server's geometry (its defaults unless --k / --seg-rows fix it)
    k_srv = a.k or 4
    seg_srv = a.seg_rows if (a.seg_rows and a.workload == "serve") else 96
    geo = binding.config(kernel=binding.SDFG_KERNEL_PERSISTENT, k=k_srv, seg_rows=seg_srv, warps=4)

    def serve(arrivals):
        sv = ctypes.c_void_p()
        binding.check(L.sdfg_server_create(ctypes.byref(sv), budget, 1024, quantum, stride, 0))
        binding.check(L.sdfg_server_set_config(sv, ctypes.byref(geo)))
        ids = [None] * n
        t0 = time.perf_counter()

        def submitter():
            for i in np.argsort(arrivals, kind="stable"):
                dt = t0 + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                d = binding.desc_for(xs[i], ys[i], cap, tol)
                rid = ctypes.c_uint64()
                binding.check(L.sdfg_server_submit(sv, ctypes.byref(d), ctypes.byref(rid)))
                ids[i] = rid.value

        th = threading.Thread(target=submitter)
        th.start()
        done_t = [None] * n
        steps = [0] * n
        res = binding.sdfg_desc()
        left = n
        pending, scanned = [], 0
        order = list(np.argsort(arrivals, kind="stable"))
        while left:
            while scanned < n and ids[order[scanned]] is not None:
                pending.append(order[scanned])
                scanned += 1
            still = []
            for i in pending:
                rc = L.sdfg_server_poll(sv, ids[i], ctypes.byref(res))
                if rc == binding.SDFG_PENDING:
                    still.append(i)
                    continue
                binding.check(rc)
                done_t[i] = time.perf_counter()
                steps[i] = res.steps_done
                left -= 1
            pending = still
            time.sleep(0.001)
        th.join()
        binding.check(L.sdfg_server_destroy(sv))
        lat = [done_t[i] - (t0 + arrivals[i]) for i in range(n)]
        span = max(done_t) - t0
        return lat, steps, span

    def plain(arrivals, limit_s):
        """One blocking solve per request in arrival order, until `limit_s` of
        wall time; returns the served prefix only."""
        t0 = time.perf_counter()
        lat, steps, idx, done = [], [], [], 0.0
        for i in np.argsort(arrivals, kind="stable"):
            if time.perf_counter() - t0 > limit_s:
                break
            dt = t0 + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            d = binding.desc_for(xs[i], ys[i], cap, tol)
            binding.check(binding.sdfg_jacobi2d_solve(d, stride, geo))
            done = time.perf_counter()
            lat.append(done - (t0 + arrivals[i]))
            steps.append(d.steps_done)
            idx.append(int(i))
        return lat, steps, done - t0, idx

    def gups(steps, span, idx=None):
        sel = [reqs[i] for i in idx] if idx is not None else reqs
        return sum((r.rows - 2) * (r.cols - 2) * s for r, s in zip(sel, steps)) / span / 1e9

    # capacity: everything queued at t = 0
    lat0, steps0, span0 = serve(np.zeros(n))
    capacity = n / span0
    rate = rho * capacity
    arrivals = inputs.poisson_arrivals(n, rate, seed=1)
    lat_s, steps_s, span_s = serve(arrivals)
    lat_p, steps_p, span_p, idx_p = plain(arrivals, plain_seconds)
    # the server's latencies on the same prefix of the trace, for a like-for-like comparison
    lat_s_prefix = [lat_s[i] for i in idx_p]
    del xs, ys
    torch.cuda.empty_cache()
    return {
        "workload": f"served_laplace_first{n}of10000req_32to4096_tol1e-6_cap20000_f32",
        "requests": n, "capacity_req_per_s": capacity, "capacity_gupdates": gups(steps0, span0), "rho": rho,
        "arrival_rate_hz": rate,
        "server": {"p50_s": _pct(lat_s, 50), "p99_s": _pct(lat_s, 99), "gupdates": gups(steps_s, span_s),
                   "makespan_s": span_s},
        "plain_launches": {"p50_s": _pct(lat_p, 50), "p99_s": _pct(lat_p, 99),
                           "gupdates": gups(steps_p, span_p, idx_p), "requests_served": len(idx_p),
                           "wall_cap_s": plain_seconds},
        "server_on_same_prefix": {"p50_s": _pct(lat_s_prefix, 50), "p99_s": _pct(lat_s_prefix, 99),
                                  "requests": len(idx_p)},
        "steps_equal_server_vs_plain": sum(int(steps_s[i] == s_) for i, s_ in zip(idx_p, steps_p)),
        "budget_bytes": budget, "quantum_steps": quantum, "check_stride": stride,
        "geometry": {"k": k_srv, "seg_rows": seg_srv, "kernel": "persistent",
                     "note": "server and plain launches run the same units, so every request stops at the "
                             "same step on both paths"},
    }


def run_serve(a):
    print(json.dumps({"metric": METRIC, "unit": UNIT, **measure_serve(a, a.requests, a.rho, a.plain_seconds)}))


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "precision":
        run_precision(a)
    elif a.workload == "serve":
        run_serve(a)
    elif a.workload == "3d":
        run_3d(a)
    elif a.workload == "sor":
        run_sor(a)
    elif a.workload == "paper":
        run_paper(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
