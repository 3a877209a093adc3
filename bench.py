#!/usr/bin/env python3
"""Benchmark: exact DTW (ParDTW) throughput in GCUPS on GB300.

One step = one exact alignment of the 20000x12 vs 25000x12 chroma-like pair
(normalise, column-sweep DP with on-the-fly cosine cost, band entry map,
band chain, band walks, path emit: 6 kernels), with the inputs already
resident in HBM.  GCUPS = La*Lb / t / 1e9.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU; a single pair does not shard
(its DP is one wavefront), so every rank aligns its own replica pair and
the value is the sum over ranks (weak scaling, replicas only).

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload (there is no reference code
to install: the paper's repository is not available here).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact DTW GCUPS on 1 GB300; learned-band speedup at <=1-frame path error"
UNIT = "GCUPS"
WORKLOAD = "pair-20000x12-vs-25000x12 chroma-like, warped (64 knots, tempo 0.7-1.4), cosine cost"
L2_FLUSH_BYTES = 512 << 20
KERNELS_PER_STEP = 6  # normalise, DP, band map, band chain, band walks, emit
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def workload_name(La, Lb):
    if (La, Lb) == (20000, 25000):
        return WORKLOAD
    return f"pair-{La}x12-vs-{Lb}x12 chroma-like, warped (64 knots, tempo 0.7-1.4), cosine cost"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.window = None

    def __enter__(self):
        # started before the timed region (nvidia-smi takes a moment to begin
        # sampling); only samples read between mark_start and mark_end count
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.time() + 3.0
            while not self.lines and time.time() < deadline:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark_start(self):
        self.window = [time.time(), None]

    def mark_end(self):
        if self.window:
            self.window[1] = time.time()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.window if self.window and self.window[1] else (0.0, float("inf"))
        # a sample arrives after its 20 ms interval: keep the ones taken inside
        for ts, ln in self.lines:
            if not (t0 < ts <= t1 + 0.02):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


DP_SOURCES = ("paper_2607_15478_gb300/csrc/dp_split.cu", "paper_2607_15478_gb300/csrc/dp_device.cuh",
              "paper_2607_15478_gb300/csrc/pardtw_common.cuh")


def dp_sources_sha256():
    """One hash over the sources the timed DP kernel is built from."""
    import hashlib
    h = hashlib.sha256()
    for rel in DP_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def dp_traffic_from_profiles():
    """DRAM bytes per DP launch from the committed ncu summary, if it matches the source."""
    p = os.path.join(ROOT, "profiles", "dp_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("source_sha256") != dp_sources_sha256():
            return None
        return float(d["dram_bytes_per_launch_full"])
    except Exception:
        return None


def oracle_sample(wp, cells_target=None):
    """Time the FP64 oracle single-threaded on the leading block of the pair."""
    import oracle
    La, Lb = wp.A.shape[0], wp.B.shape[0]
    if cells_target is None:
        a, b = La, Lb
    else:
        s = min(1.0, (cells_target / (La * Lb)) ** 0.5)
        a, b = max(2, int(La * s)), max(2, int(Lb * s))
    A, B = wp.A[:a], wp.B[:b]
    t0 = time.perf_counter()
    oracle.dtw(A, B)
    dt = time.perf_counter() - t0
    return a, b, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2607_15478_gb300 import synth
    import oracle
    oracle.build()
    wp = synth.config_pair(1)
    cells_target = 1.0e8  # ~2 s of single-threaded FP64 work per step
    times, cells = [], 0
    for k in range(args.warmup + args.steps):
        a, b, dt = oracle_sample(wp, cells_target)
        if k >= args.warmup:
            times.append(dt)
            cells = a * b
    t = sum(times)
    v = cells * len(times) / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "La": 20000, "Lb": 25000, "D": 12},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"leading {a}x{b} block of the pair per step, single-threaded "
                                   f"FP64 row-by-row DTW"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local if ws > 1 else 0)
    from paper_2607_15478_gb300 import build as pbuild
    if rank == 0 or ws == 1:
        pbuild.build()
    if ws > 1:
        dist.barrier()
    from paper_2607_15478_gb300 import pardtw, synth

    wp = synth.config_pair(1, pair=rank, La=args.La, Lb=args.Lb)
    La, Lb, D = wp.A.shape[0], wp.B.shape[0], wp.A.shape[1]
    cells = La * Lb
    stream = torch.cuda.Stream(device=dev)
    al = pardtw.Aligner(dev.index, stream)
    al.enable_timing(True)
    A = torch.from_numpy(wp.A).to(dev)
    B = torch.from_numpy(wp.B).to(dev)
    cap = min(La, Lb)
    path = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    plen = torch.zeros(1, dtype=torch.int32, device=dev)
    tot = torch.zeros(1, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1)          # L2 flush, outside the events
            ev0.record(stream)
            al.align_into(A, B, path, plen, tot)
            ev1.record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    n_ok = int(plen.item())
    if n_ok <= 0:
        raise RuntimeError(f"alignment failed on rank {rank}: {pardtw.status_string(-n_ok)}")

    step_ms, dp_ms = [], []
    with ClockSampler(dev.index) as clk:  # sampling starts before the barrier
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clk.mark_start()
        for _ in range(args.steps):
            step()
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            dp_ms.append(al.stage_times()[1])
        torch.cuda.synchronize(dev)
        clk.mark_end()
        if ws > 1:
            dist.barrier()
    t_local = sum(step_ms) / 1e3
    if ws > 1:
        t = torch.tensor([t_local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    else:
        t_max = t_local
    value = ws * cells * args.steps / t_max / 1e9

    # end to end through the public API with host buffers: H2D of A and B,
    # alignment, D2H of path, length and total inside the timed region
    Ah = torch.from_numpy(wp.A).pin_memory()
    Bh = torch.from_numpy(wp.B).pin_memory()
    ph = torch.empty((cap, 2), dtype=torch.int32).pin_memory()
    lh = torch.zeros(1, dtype=torch.int32).pin_memory()
    th = torch.zeros(1, dtype=torch.float32).pin_memory()
    al.enable_timing(False)
    e2e_t = []
    for k in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        t0 = time.perf_counter()
        pardtw.dtw_align(al.h, Ah, Bh, ph, lh, th)
        e2e_t.append(time.perf_counter() - t0)
    e2e_t = e2e_t[args.warmup:]
    t_e2e = sum(e2e_t)
    if ws > 1:
        t = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())
    e2e_value = ws * cells * args.steps / t_e2e / 1e9
    h2d = (La + Lb) * D * 4
    d2h = int(lh[0]) * 8 + 8

    if rank == 0:
        peaks, src = measured_peaks()
        clock = peaks.get("sm_max_mhz", 2070.0)
        peak_ops = SM_COUNT * FP32_LANES_PER_SM * clock * 1e6      # FP32 lane-ops/s
        ops_per_cell = D + 6
        dp_avg = statistics.mean(dp_ms) / 1e3
        achieved = cells * ops_per_cell / dp_avg
        traffic = dp_traffic_from_profiles()
        cpu = None
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            a, b, dt = oracle_sample(wp)
            cpu = {"value": a * b / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"the full {a}x{b} pair once, single-threaded FP64 row-by-row DTW "
                             f"({dt:.1f} s)"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(La, Lb), "La": La, "Lb": Lb, "D": D,
                       "l2": "flushed between steps (512 MiB write)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "T FP32 lane-ops/s", "frac": achieved / peak_ops,
                         "traffic": traffic,
                         "kernel": "k_dp_split (column-sweep DP: per strip a cost warp and a DP "
                                   "warp, cost on the fly)",
                         "ops_per_cell": ops_per_cell, "dp_ms": 1e3 * dp_avg,
                         "peak_basis": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                       f"{clock:.0f} MHz (sm_max_mhz, {src})"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": KERNELS_PER_STEP * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    al.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--La", type=int, default=None,
                    help="override the pair's lengths (same recipe; for profiling smaller cases)")
    ap.add_argument("--Lb", type=int, default=None)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
