#!/usr/bin/env python3
"""Benchmark: exact DTW (ParDTW) throughput in GCUPS on GB300.

One step = one exact alignment of the 20000x12 vs 25000x12 chroma-like pair
(normalise, column-sweep DP with on-the-fly cosine cost, band entry map,
two- and four-band maps, band chain, band walks, path emit: 8 kernels), with the inputs
already resident in HBM.  GCUPS = La*Lb / t / 1e9.

The same JSON line carries the second half of the metric and the project's
other forms, each measured in this run on this GPU: a `band` block (the
100000 x 126231 pair in the learned band against the full exact DP: speedup,
fallbacks, path deviation), a `batch` block (256 uneven pairs as one CUDA
graph), a `bf16` block (the 40000x128 vs 48000x128 pair, BF16 cost on the
tensor cores against the FP32 cost) and a `cost_matrix` block (the explicit
cost matrix of the default pair through dtw_cost: GB/s written).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config 1..5] [--no-extras]

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


def backtrace_kernels(rows):
    """Launches of the parallel backtrace of a sweep with `rows` rows: band
    map, two-band map (at least 4 bands of 128 rows), four-band map (at least
    6), chain, walks, emission.  Every workload here has at least 768 frames on
    each side, so both sweep directions give the same count."""
    nb = -(-rows // 128)
    return 4 + (nb >= 4) + (nb >= 6)


# normalise, DP, backtrace
KERNELS_PER_STEP = 2 + backtrace_kernels(20000)
# learned band: 2 x (pool, 3 convolutions, heads), coarse alignment of the
# 8x pooled sequences (normalise, DP, backtrace), band ranges (2), banded
# alignment (normalise, DP, backtrace), band-side test (1)
KERNELS_PER_LEARNED_STEP = 10 + (2 + backtrace_kernels(100000 // 8)) + 2 + (2 + backtrace_kernels(100000)) + 1
# WSDTW: batched normalisation, subsequence DP, segment DP (one cooperative
# launch while every column tile's CTA fits on the GPU at once, as at this
# size; else a tile pass and a fix-up pass per fragment), fragment
# backtraces, compaction
def kernels_per_wsdtw_step(nfrag, Lb):
    return 5 if (Lb + 1023) // 1024 <= 2 * SM_COUNT else 4 + 2 * nfrag
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


def step_stats(ms):
    """Median, 10th and 90th percentile of per-step times (ms)."""
    import numpy as np
    a = np.asarray(ms, dtype=np.float64)
    return {"median": float(np.median(a)), "p10": float(np.percentile(a, 10)),
            "p90": float(np.percentile(a, 90)), "n": int(a.size)}


def cpu_info():
    """Host cores and CPU model of the machine the oracle is timed on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu model")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown",
            "machine": os.uname().machine}


def jbar(pp, n):
    """Mean column matched to each row, interpolated over rows a (2,1) step skips."""
    import numpy as np
    acc, cnt = np.zeros(n), np.zeros(n)
    np.add.at(acc, pp[:, 0], pp[:, 1])
    np.add.at(cnt, pp[:, 0], 1)
    rows = np.flatnonzero(cnt)
    return np.interp(np.arange(n), rows, acc[rows] / cnt[rows])


def mean_path_deviation(p, q, La):
    import numpy as np
    return float(np.mean(np.abs(jbar(p, La) - jbar(q, La))))


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
                 "--format=csv,noheader,nounits", "-lms", "5"],
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
        # a sample arrives after its 5 ms interval: keep the ones taken inside
        for ts, ln in self.lines:
            if not (t0 < ts <= t1 + 0.005):
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


DP_SOURCES = ("paper_2607_15478_gb300/csrc/dp_split.cuh", "paper_2607_15478_gb300/csrc/dp_split.cu",
              "paper_2607_15478_gb300/csrc/dp_split_cl.cu", "paper_2607_15478_gb300/csrc/dp_split_cl.cuh",
              "paper_2607_15478_gb300/csrc/dp_device.cuh")


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
                                   f"FP64 row-by-row DTW", **cpu_info()},
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

    step_ms, dp_ms, stages = [], [], []
    with ClockSampler(dev.index) as clk:  # sampling starts before the barrier
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clk.mark_start()
        for _ in range(args.steps):
            step()
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            st = al.stage_times()
            stages.append(st)
            dp_ms.append(st[1])
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
    d2h = cap * 8 + 8  # total and length, and the path buffer's min(La, Lb) pairs

    al.close()
    if rank == 0:
        peaks, src = measured_peaks()
        nominal_ops, basis = nominal_peak(peaks, src)
        # the FP32 FMA rate measured on this GPU in this run (an FFMA counts as
        # one lane-op, as the D dot-product FMAs of a cell do)
        with ClockSampler(dev.index) as pclk:
            pclk.mark_start()
            peak_ops = pardtw.fp32_peak(dev.index)
            pclk.mark_end()
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
                             f"({dt:.1f} s)", **cpu_info()}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "step_ms": step_stats(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(La, Lb), "La": La, "Lb": Lb, "D": D,
                       "l2": "flushed between steps (512 MiB write)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "T FP32 lane-ops/s", "frac": achieved / peak_ops,
                         "traffic": traffic,
                         "kernel": "k_dp_split (column-sweep DP: per strip a cost warp and a DP "
                                   "warp, cost on the fly; thread-block clusters, the strip "
                                   "border between CTAs of a cluster in distributed shared "
                                   "memory)",
                         "ops_per_cell": ops_per_cell, "dp_ms": 1e3 * dp_avg,
                         "dp_launch_ms": step_stats(dp_ms),
                         "peak_basis": "FFMA rate measured in this run (dtw_fp32_peak: every SM "
                                       "sub-partition issuing independent FFMAs)",
                         "peak_clocks": pclk.summary(),
                         "nominal_peak": nominal_ops / 1e12, "nominal_basis": basis,
                         "frac_of_nominal": achieved / nominal_ops},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": KERNELS_PER_STEP * args.steps,
            "stage_ms": {
                "normalise": statistics.median(x[0] for x in stages),
                "dp": statistics.median(x[1] for x in stages),
                "backtrace": statistics.median(x[2] for x in stages),
                "timing": "CUDA events around each stage on the aligner's stream; medians "
                          "over the timed steps"},
            "clocks": clk.summary(),
        }
        if ws == 1 and not args.no_extras:
            # the metric's second half and the other forms, on this GPU in this
            # run: each block times its own workload (CUDA events, medians)
            k = max(5, min(args.steps, 20))
            line["band"], ex = measure_band(dev, k, args.warmup, flush)
            ex["al"].close()
            line["batch"], ex = measure_batch(dev, k, args.warmup, flush)
            ex["plan"].close()
            ex["al"].close()
            line["bf16"], ex = measure_bf16(dev, k, args.warmup, flush)
            ex["al"].close()
            line["cost_matrix"], ex = measure_cost(dev, k, args.warmup)
            ex["al"].close()
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _rank0_line(line):
    print(json.dumps(line), flush=True)


def measure_cost(dev, steps, warmup):
    """The explicit cost matrix of the 20000x12 vs 25000x12 pair through
    dtw_cost (an inspection surface: the aligner never stores it): 4 bytes
    written a cell, so HBM-bound.  2.0 GB, larger than L2: no flush needed."""
    import torch
    from paper_2607_15478_gb300 import pardtw, synth
    wp = synth.config_pair(1)
    La, Lb, D = wp.A.shape[0], wp.B.shape[0], wp.A.shape[1]
    stream = torch.cuda.Stream(device=dev)
    al = pardtw.Aligner(dev.index, stream)
    A = torch.from_numpy(wp.A).to(dev)
    B = torch.from_numpy(wp.B).to(dev)
    C = torch.empty((La, Lb), dtype=torch.float32, device=dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def step():
        with torch.cuda.stream(stream):
            ev0.record(stream)
            pardtw.dtw_cost(al.h, A, B, C)
            ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    for _ in range(warmup):
        step()
    ms = [step() for _ in range(steps)]
    med = statistics.median(ms)
    written = La * Lb * 4
    peaks, basis = measured_peaks()
    gbs = written / med / 1e6
    block = {
        "workload": workload_name(La, Lb) + ", La x Lb float32 matrix",
        "ms": med, "step_ms": step_stats(ms), "gcups": La * Lb / med / 1e6,
        "bytes_written": written, "gbs": gbs, "peak_gbs": peaks["hbm_gbs"],
        "frac_of_hbm": gbs / peaks["hbm_gbs"],
        "peak_basis": f"HBM copy bandwidth ({basis})",
        "kernels": "k_normalise + k_cost (4 x 4 cells a thread, b^ of its 4 columns in registers over its row tiles, one 16-byte store per row of 4)",
        "timing": "CUDA events on the aligner's stream, device buffers",
    }
    del C
    return block, {"al": al}


def measure_band(dev, steps, warmup, flush, exact_runs=3):
    """The learned-band workload (the 100000x12 vs 126231x12 pair, tempo
    0.6-1.6, 256 knots) aligned exactly inside the band of the trained
    encoder (dtw_align_learned, bf16 encoder) and, on the same GPU in the same
    run, by the full exact DP.  Returns the block and what the --config 4 line
    adds (timings of the banded DP launches, clocks, the pair)."""
    import numpy as np
    import torch
    from paper_2607_15478_gb300 import band_train, pardtw, synth
    wp = synth.config_pair(4)
    La, Lb = wp.A.shape[0], wp.B.shape[0]
    stream = torch.cuda.Stream(device=dev)
    al = pardtw.Aligner(dev.index, stream)
    al.enable_timing(True)
    P = band_train.load(device=dev)
    A = torch.from_numpy(wp.A).to(dev)
    B = torch.from_numpy(wp.B).to(dev)
    cap = min(La, Lb)
    path = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    plen = torch.zeros(1, dtype=torch.int32, device=dev)
    tot = torch.zeros(1, dtype=torch.float32, device=dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    fell = []

    def step(exact=False):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            ev0.record(stream)
            if exact:
                al.align_into(A, B, path, plen, tot)
            else:
                fell.append(pardtw.dtw_align_learned(al.h, A, B, P, path, plen, tot, 8, True))
            ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    for _ in range(2):
        step(exact=True)
    exact_all = [step(exact=True) for _ in range(exact_runs)]
    if int(plen.item()) <= 0:
        raise RuntimeError(f"exact alignment failed: {pardtw.status_string(-int(plen.item()))}")
    p_exact = path[:int(plen.item())].cpu().numpy()
    t_exact = float(tot.item())
    for _ in range(warmup):
        step()
    fell.clear()
    step_ms, dp_ms = [], []
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        clk.mark_start()
        for _ in range(steps):
            step_ms.append(step())
            dp_ms.append(al.stage_times()[1])
        clk.mark_end()
    if int(plen.item()) <= 0:
        raise RuntimeError(f"banded alignment failed: {pardtw.status_string(-int(plen.item()))}")
    band_cells = al.band_cells()
    p_band = path[:int(plen.item())].cpu().numpy()
    t_band = float(tot.item())
    exact_ms = statistics.median(exact_all)
    band_ms = statistics.median(step_ms)
    block = {
        "workload": f"pair-{La}x12-vs-{Lb}x12 chroma-like, warped (256 knots, tempo 0.6-1.6)",
        "exact_ms": exact_ms, "band_ms": band_ms, "speedup_vs_exact": exact_ms / band_ms,
        "band_step_ms": step_stats(step_ms), "exact_step_ms": step_stats(exact_all),
        "fell_back_steps": int(sum(fell)), "steps": steps,
        "same_path_as_exact": bool(p_band.shape == p_exact.shape and
                                   np.array_equal(p_band, p_exact)),
        "mean_path_deviation_frames": mean_path_deviation(p_band, p_exact, La),
        "total_rel_diff_vs_exact": abs(t_band - t_exact) / abs(t_exact),
        "band_cells": band_cells, "band_fraction": band_cells / (La * Lb),
        "exact_gcups": La * Lb / exact_ms / 1e6,
        "weights": "paper_2607_15478_gb300/weights/band_encoder_d12.npy",
        "timing": "CUDA events on the aligner's stream, L2 flushed before every step; "
                  "medians over the steps",
    }
    extra = {"wp": wp, "al": al, "P": P, "stream": stream, "step_ms": step_ms,
             "dp_ms": dp_ms, "clocks": clk.summary()}
    return block, extra


def measure_batch(dev, steps, warmup, flush, pairs=None, want_e2e=False):
    """The batching workload: 256 seeded pairs (La ~ U[500, 8000], Lb = La x
    U[0.8, 1.25], D = 12) as a planned batch (dtw_batch_create: DP schedule
    picked by the autotuner, the whole batch captured in one CUDA graph); a
    step is one graph replay.  The same batch through dtw_align_many (no
    graph) is timed beside it."""
    import numpy as np
    import torch
    from paper_2607_15478_gb300 import pardtw, synth
    if pairs is None:
        pairs = synth.config_batch(2)
    cells = sum(p.A.shape[0] * p.B.shape[0] for p in pairs)
    stream = torch.cuda.Stream(device=dev)
    al = pardtw.Aligner(dev.index, stream)
    al.enable_timing(True)
    # all features in one device buffer (A of every pair, then B of every
    # pair), the pairs' inputs being views of it, so that one host-to-device
    # copy refills a whole batch
    sizes = [p.A.size for p in pairs] + [p.B.size for p in pairs]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    feat_h = torch.empty(int(offs[-1]), dtype=torch.float32).pin_memory()
    for k, x in enumerate([p.A for p in pairs] + [p.B for p in pairs]):
        feat_h[int(offs[k]):int(offs[k + 1])] = torch.from_numpy(x.reshape(-1))
    feat = feat_h.to(dev)
    n_p = len(pairs)
    As = [feat[int(offs[k]):int(offs[k + 1])].view(pairs[k].A.shape) for k in range(n_p)]
    Bs = [feat[int(offs[n_p + k]):int(offs[n_p + k + 1])].view(pairs[k].B.shape)
          for k in range(n_p)]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    st = None

    def step_many():
        nonlocal st
        with torch.cuda.stream(stream):
            flush.fill_(1)
            ev0.record(stream)
            _, _, st = al.align_many(As, Bs)
            ev1.record(stream)

    many_ms, dp_ms = [], []
    for k in range(warmup + 3):
        step_many()
        ev1.synchronize()
        if k >= warmup:
            many_ms.append(ev0.elapsed_time(ev1))
            dp_ms.append(al.stage_times()[1])
    if st is not None and (st != 0).any():
        raise RuntimeError("batch alignment failed")
    plan = al.plan_batch(As, Bs, autotune=True)
    R_tuned, NS_tuned, tuned_ms = plan.info()

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1)
            ev0.record(stream)
            plan.run()
            ev1.record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    if (plan.path_len.cpu().numpy() <= 0).any():
        raise RuntimeError("planned batch failed")
    step_ms = []
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        clk.mark_start()
        for _ in range(steps):
            step()
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
        torch.cuda.synchronize(dev)
        clk.mark_end()
    graph_ms = statistics.median(step_ms)
    block = {
        "workload": "batch-256-pairs La~U[500,8000] Lb=La*U[0.8,1.25] D=12 chroma-like, "
                    "warped (8 knots)" if n_p == 256 else f"batch of {n_p} pairs",
        "pairs": n_p, "cells": cells, "graph_ms": graph_ms, "gcups": cells / graph_ms / 1e6,
        "graph_step_ms": step_stats(step_ms), "align_many_ms": statistics.median(many_ms),
        "align_many_dp_ms": statistics.median(dp_ms),
        "autotune_rows_per_lane": R_tuned, "autotune_strips_per_cta": NS_tuned,
        "autotune_ms": {f"R{r}_NS{ns}": tuned_ms[(3 if ns == 4 else 0) + r - 2]
                        for ns in (2, 4) for r in (2, 3, 4)},
        "timing": "CUDA events around one graph replay, L2 flushed before every step",
    }
    extra = {"step_ms": step_ms, "dp_ms": dp_ms, "clocks": clk.summary(), "plan": plan,
             "al": al, "stream": stream, "feat": feat, "feat_h": feat_h}
    if want_e2e:
        # end to end: the batch's features copied in from pinned host memory
        # (one copy into the plan's input buffer), the plan's graph, paths,
        # lengths and costs copied out (one copy each), split per pair
        paths_h = torch.empty(plan.paths.shape, dtype=torch.int32).pin_memory()
        lens_h = torch.empty(plan.path_len.shape, dtype=torch.int32).pin_memory()
        cost_h = torch.empty(plan.cost.shape, dtype=torch.float32).pin_memory()
        al.enable_timing(False)
        e2e_t = []
        for k in range(warmup + steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            stream.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                feat.copy_(feat_h, non_blocking=True)
                plan.run()
                paths_h.copy_(plan.paths, non_blocking=True)
                lens_h.copy_(plan.path_len, non_blocking=True)
                cost_h.copy_(plan.cost, non_blocking=True)
            stream.synchronize()
            ln = lens_h.numpy()
            _ = [paths_h[int(plan.off[q]):int(plan.off[q]) + int(ln[q])] for q in range(n_p)]
            e2e_t.append(time.perf_counter() - t0)
        extra["e2e_s"] = sum(e2e_t[warmup:])
        extra["h2d"] = int(feat_h.numel()) * 4
        extra["d2h"] = int(paths_h.numel()) * 4 + 8 * n_p
    return block, extra


def measure_bf16(dev, steps, warmup, flush, fp32_runs=2, La=None, Lb=None):
    """The precision workload: the 40000x128 vs 48000x128 pair with the cost
    from bf16 features on the tensor cores (FP32 accumulate, FP32 DP), against
    the FP32 cost path on the same GPU in the same run."""
    import torch
    from paper_2607_15478_gb300 import pardtw, synth
    wp = synth.config_pair(3, La=La, Lb=Lb)
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
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def step(prec):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            ev0.record(stream)
            al.align_into(A, B, path, plen, tot, cost_precision=prec)
            ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    for _ in range(warmup):
        step(1)
    step_ms, dp_ms = [], []
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        clk.mark_start()
        for _ in range(steps):
            step_ms.append(step(1))
            dp_ms.append(al.stage_times()[1])
        clk.mark_end()
    if int(plen.item()) <= 0:
        raise RuntimeError(f"bf16 alignment failed: {pardtw.status_string(-int(plen.item()))}")
    tot_bf, path_bf = float(tot.item()), path[:int(plen.item())].cpu().numpy()
    step(0)  # warm-up of the FP32 cost path
    fp32_all, fp32_dp = [], []
    for _ in range(fp32_runs):
        fp32_all.append(step(0))
        fp32_dp.append(al.stage_times()[1])
    tot_f32, path_f32 = float(tot.item()), path[:int(plen.item())].cpu().numpy()
    bf16_ms = statistics.median(step_ms)
    fp32_ms = statistics.median(fp32_all)
    block = {
        "workload": f"pair-{La}x128-vs-{Lb}x128 gaussian frames, L2-normalised, warped "
                    "(64 knots) + N(0,0.1)",
        "bf16_ms": bf16_ms, "bf16_gcups": cells / bf16_ms / 1e6,
        "bf16_step_ms": step_stats(step_ms), "bf16_dp_ms": statistics.median(dp_ms),
        "fp32_ms": fp32_ms, "fp32_gcups": cells / fp32_ms / 1e6,
        "fp32_dp_ms": statistics.median(fp32_dp),
        "speedup_vs_fp32_cost": fp32_ms / bf16_ms,
        "total_rel_diff_vs_fp32": abs(tot_bf - tot_f32) / abs(tot_f32),
        "mean_path_deviation_vs_fp32_frames": mean_path_deviation(path_bf, path_f32, La),
        "error_vs_fp64_oracle": "tests/test_gpu_bf16.py (recorded in profiles/)",
        "timing": "CUDA events on the aligner's stream, L2 flushed before every step",
    }
    extra = {"wp": wp, "al": al, "stream": stream, "step_ms": step_ms, "dp_ms": dp_ms,
             "clocks": clk.summary(), "cells": cells}
    return block, extra


def nominal_peak(peaks, src):
    clock = peaks.get("sm_max_mhz", 2070.0)
    return (SM_COUNT * FP32_LANES_PER_SM * clock * 1e6,
            f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x {clock:.0f} MHz "
            f"(sm_max_mhz, {src})")


def run_batch(args):
    """--config 2: the batching workload's own line (strong scaling: N ranks
    split the 256 pairs by cell count, LPT, and align their shares)."""
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
    from paper_2607_15478_gb300 import shard, synth
    pairs_all = synth.config_batch(2)
    cells_all = [p.A.shape[0] * p.B.shape[0] for p in pairs_all]
    mine = shard.partition_pairs(cells_all, ws)[rank]
    pairs = [pairs_all[k] for k in mine]
    cells = sum(cells_all[k] for k in mine)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    if ws > 1:
        dist.barrier()
    block, ex = measure_batch(dev, args.steps, args.warmup, flush, pairs=pairs, want_e2e=True)
    t_local = sum(ex["step_ms"]) / 1e3
    t_max, t_e2e = t_local, ex["e2e_s"]
    if ws > 1:
        t = torch.tensor([t_local, t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max, t_e2e = float(t[0].item()), float(t[1].item())
    value = sum(cells_all) * args.steps / t_max / 1e9
    if rank == 0:
        peaks, src = measured_peaks()
        peak_ops, basis = nominal_peak(peaks, src)
        dp_avg = statistics.mean(ex["dp_ms"]) / 1e3
        achieved = cells * 18 / dp_avg
        cpu = None
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            t0 = time.perf_counter()
            done = 0
            for p in pairs_all:
                if time.perf_counter() - t0 > 15.0:
                    break
                oracle.dtw(p.A, p.B)
                done += p.A.shape[0] * p.B.shape[0]
            dt = time.perf_counter() - t0
            cpu = {"value": done / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"the first pairs of the batch, one after another, until 15 s "
                             f"({done / 1e9:.2f} Gcells in {dt:.1f} s), single-threaded FP64",
                   **cpu_info()}
        _rank0_line({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "step_ms": step_stats(ex["step_ms"]),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batch-256-pairs La~U[500,8000] Lb=La*U[0.8,1.25] D=12 "
                                   "chroma-like, warped (8 knots)",
                       "pairs": len(pairs_all), "cells": sum(cells_all), "D": 12,
                       "l2": "flushed between steps (512 MiB write)",
                       "parallelism": f"pairs split by cell count over {ws} rank(s)",
                       "graph": "one CUDA graph replay per step (dtw_batch_run)",
                       "schedule": f"autotuned: {block['autotune_rows_per_lane']} rows per "
                                   f"lane, {block['autotune_strips_per_cta']} strips per CTA"},
            "batch": block,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "T FP32 lane-ops/s", "frac": achieved / peak_ops,
                         "traffic": None,
                         "kernel": "k_dp_split, batch mode (work queue over pairs), timed "
                                   "through dtw_align_many",
                         "ops_per_cell": 18, "dp_ms": 1e3 * dp_avg, "peak_basis": basis},
            "cpu_baseline": cpu,
            "e2e": {"value": sum(cells_all) * args.steps / t_e2e / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": ex["h2d"], "d2h_bytes_per_step": ex["d2h"]},
            # epoch bump, normalisation, DP, backtrace (bands over the longest A)
            "gpu_launches": (3 + backtrace_kernels(max((p.A.shape[0] for p in pairs), default=0)))
                            * args.steps,
            "clocks": ex["clocks"],
        })
    ex["plan"].close()
    ex["al"].close()
    if ws > 1:
        dist.destroy_process_group()


def run_precision(args):
    """--config 3: the precision workload's own line."""
    import torch
    ws, rank, local = dist_env()
    dev = torch.device("cuda", local if ws > 1 else 0)
    from paper_2607_15478_gb300 import build as pbuild
    pbuild.build()
    from paper_2607_15478_gb300 import pardtw
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    block, ex = measure_bf16(dev, args.steps, args.warmup, flush, La=args.La, Lb=args.Lb)
    wp, al, cells = ex["wp"], ex["al"], ex["cells"]
    La, Lb, D = wp.A.shape[0], wp.B.shape[0], wp.A.shape[1]
    cap = min(La, Lb)
    t = sum(ex["step_ms"]) / 1e3
    # e2e: host features in, path out
    Ah = torch.from_numpy(wp.A).pin_memory()
    Bh = torch.from_numpy(wp.B).pin_memory()
    ph = torch.empty((cap, 2), dtype=torch.int32).pin_memory()
    lh = torch.zeros(1, dtype=torch.int32).pin_memory()
    th = torch.zeros(1, dtype=torch.float32).pin_memory()
    al.enable_timing(False)
    opts = pardtw.make_options(cost_precision=1)
    e2e_t = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pardtw.dtw_align(al.h, Ah, Bh, ph, lh, th, opts)
        e2e_t.append(time.perf_counter() - t0)
    t_e2e = sum(e2e_t[args.warmup:])
    peaks, src = measured_peaks()
    dp_avg = statistics.mean(ex["dp_ms"]) / 1e3
    tflops = cells * 2 * 128 / dp_avg / 1e12
    peak_tf = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
    _rank0_line({
        "metric": METRIC, "value": cells * args.steps / t / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "step_ms": step_stats(ex["step_ms"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 cost (f32 accumulate), f32 DP",
        "data": "synthetic",
        "config": {"workload": block["workload"], "La": La, "Lb": Lb, "D": D,
                   "l2": "flushed between steps (512 MiB write)", "parallelism": "single GPU"},
        "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak_tf,
                     "unit": "TFLOP/s", "frac": tflops / peak_tf, "traffic": None,
                     "kernel": "k_dp_split BF16 (cost warps: mma.sync m16n8k16; DP warps FP32)",
                     "dp_ms": 1e3 * dp_avg,
                     "note": "cost contraction flops (2 x 128 per cell) over the DP launch; the "
                             "launch is bound by the DP recurrence, not the tensor pipe"},
        "bf16": block,
        "cpu_baseline": None,
        "e2e": {"value": cells * args.steps / t_e2e / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": (La + Lb) * D * 4, "d2h_bytes_per_step": cap * 8 + 8},
        # normalisation, bf16 packing of B, DP, backtrace
        "gpu_launches": (3 + backtrace_kernels(min(La, Lb))) * args.steps,
        "clocks": ex["clocks"],
    })
    al.close()


def run_band(args):
    """--config 4: the learned-band workload's own line; value = full-matrix
    cells (La x Lb) per second of the banded alignment."""
    import torch
    ws, rank, local = dist_env()
    dev = torch.device("cuda", local if ws > 1 else 0)
    from paper_2607_15478_gb300 import build as pbuild
    pbuild.build()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    block, ex = measure_band(dev, args.steps, args.warmup, flush,
                             exact_runs=max(3, args.steps // 4))
    wp, al, P, stream = ex["wp"], ex["al"], ex["P"], ex["stream"]
    La, Lb, D = wp.A.shape[0], wp.B.shape[0], wp.A.shape[1]
    cells = La * Lb
    t = sum(ex["step_ms"]) / 1e3
    # e2e: host features in, path out, through the public API
    Ah = torch.from_numpy(wp.A).pin_memory()
    Bh = torch.from_numpy(wp.B).pin_memory()
    al.enable_timing(False)
    e2e_t = []
    for k in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            Ad = Ah.to(dev, non_blocking=True)
            Bd = Bh.to(dev, non_blocking=True)
        pth, tt, fb = al.align_learned(Ad, Bd, P)
        ph = pth.cpu()
        e2e_t.append(time.perf_counter() - t0)
    t_e2e = sum(e2e_t[args.warmup:])
    peaks, src = measured_peaks()
    peak_ops, basis = nominal_peak(peaks, src)
    ops_per_cell = D + 6
    dp_avg = statistics.mean(ex["dp_ms"]) / 1e3
    band_cells = block["band_cells"]
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        a, b, dt = oracle_sample(wp, cells_target=3.0e8)
        cpu = {"value": a * b / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"leading {a}x{b} block of the pair, single-threaded FP64 row-by-row "
                         f"exact DTW ({dt:.1f} s)", **cpu_info()}
    _rank0_line({
        "metric": METRIC, "value": cells * args.steps / t / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "step_ms": step_stats(ex["step_ms"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (encoder bf16)",
        "data": "synthetic",
        "config": {"workload": block["workload"] + ", exact DTW in the learned band",
                   "La": La, "Lb": Lb, "D": D, "downsample": 8,
                   "l2": "flushed between steps (512 MiB write)", "parallelism": "single GPU",
                   "value_definition": "La x Lb cells over the banded alignment's time"},
        "band": block,
        "roofline": {"bound": "alu", "achieved": band_cells * ops_per_cell / dp_avg / 1e12,
                     "peak": peak_ops / 1e12, "unit": "T FP32 lane-ops/s",
                     "frac": band_cells * ops_per_cell / dp_avg / peak_ops, "traffic": None,
                     "kernel": "k_dp_split over the band's strip ranges",
                     "ops_per_cell": ops_per_cell, "dp_ms": 1e3 * dp_avg, "peak_basis": basis,
                     "note": "the banded DP is one chain of strips (each waits for the "
                             "bottom rows of the one above): bound by the per-column step "
                             "latency of a strip, not by a pipe"},
        "cpu_baseline": cpu,
        "e2e": {"value": cells * args.steps / t_e2e / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": (La + Lb) * D * 4,
                "d2h_bytes_per_step": int(ph.shape[0]) * 8 + 8},
        "gpu_launches": KERNELS_PER_LEARNED_STEP * args.steps,
        "clocks": ex["clocks"],
    })
    al.close()


def run_wsdtw(args):
    """WSDTW (Sec. II-C) of the 100000x12 query against the 126231x12 reference
    of the long pair (tempo 0.6-1.6, 256 knots) with N = 32 fragments (the
    paper's setting for the Mazurka data): one batched subsequence DP over all
    fragments, the segment-level DP, the fragment backtraces.  value = La x Lb
    frame-level cells per second."""
    import numpy as np
    import torch
    ws_, rank, local = dist_env()
    dev = torch.device("cuda", local if ws_ > 1 else 0)
    from paper_2607_15478_gb300 import build as pbuild
    pbuild.build()
    from paper_2607_15478_gb300 import pardtw, synth
    wp = synth.config_pair(4, pair=rank, La=args.La, Lb=args.Lb)
    La, Lb, D = wp.A.shape[0], wp.B.shape[0], wp.A.shape[1]
    N = args.nfrag
    cells = La * Lb
    stream = torch.cuda.Stream(device=dev)
    al = pardtw.Aligner(dev.index, stream)
    al.enable_timing(True)
    A = torch.from_numpy(wp.A).to(dev)
    B = torch.from_numpy(wp.B).to(dev)
    path = torch.empty((La, 2), dtype=torch.int32, device=dev)
    plen = torch.zeros(1, dtype=torch.int32, device=dev)
    ends = torch.empty(N, dtype=torch.int32, device=dev)
    tot = torch.zeros(1, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1)
            ev0.record(stream)
            pardtw.dtw_wsdtw(al.h, A, B, N, path, plen, ends, tot)
            ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    for _ in range(args.warmup):
        step()
    if int(plen.item()) <= 0:
        raise RuntimeError(f"wsdtw failed: {pardtw.status_string(-int(plen.item()))}")
    step_ms, dp_ms = [], []
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        clk.mark_start()
        for _ in range(args.steps):
            step_ms.append(step())
            dp_ms.append(al.stage_times()[1])
        clk.mark_end()
    t = sum(step_ms) / 1e3
    value = cells * args.steps / t / 1e9
    # e2e: host features in, path out, through the public API
    Ah = torch.from_numpy(wp.A).pin_memory()
    Bh = torch.from_numpy(wp.B).pin_memory()
    al.enable_timing(False)
    e2e_t = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            Ad = Ah.to(dev, non_blocking=True)
            Bd = Bh.to(dev, non_blocking=True)
        pth, _, _ = al.wsdtw(Ad, Bd, N)
        ph = pth.cpu()
        e2e_t.append(time.perf_counter() - t0)
    t_e2e = sum(e2e_t[args.warmup:])
    peaks, src = measured_peaks()
    clock = peaks.get("sm_max_mhz", 2070.0)
    peak_ops = SM_COUNT * FP32_LANES_PER_SM * clock * 1e6
    ops_per_cell = D + 6
    dp_avg = statistics.mean(dp_ms) / 1e3
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import wsdtw as ows
        nf = 2  # two fragments of the same pair, the oracle's subsequence DP
        r0, n0 = ows.fragments(La, N)[0]
        a_rows = n0 * nf
        t0 = time.perf_counter()
        ows.wsdtw(wp.A[:a_rows], wp.B, nf)
        dt = time.perf_counter() - t0
        cpu = {"value": a_rows * Lb / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"WSDTW of the first {nf} fragments ({a_rows} rows) against all "
                         f"{Lb} frames, FP64 numpy row sweep, single thread ({dt:.1f} s)"}
    _rank0_line({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"WSDTW N={N}: query {La}x12 vs reference {Lb}x12 chroma-like, "
                               f"warped (256 knots, tempo 0.6-1.6)",
                   "La": La, "Lb": Lb, "D": D, "nfrag": N,
                   "l2": "flushed between steps (512 MiB write)", "parallelism": "single GPU",
                   "value_definition": "La x Lb frame-level cells over the step time"},
        "roofline": {"bound": "alu", "achieved": cells * ops_per_cell / dp_avg / 1e12,
                     "peak": peak_ops / 1e12, "unit": "T FP32 lane-ops/s",
                     "frac": cells * ops_per_cell / dp_avg / peak_ops, "traffic": None,
                     "kernel": "k_dp_split subsequence mode over all fragments (one launch)",
                     "ops_per_cell": ops_per_cell, "dp_ms": 1e3 * dp_avg},
        "cpu_baseline": cpu,
        "e2e": {"value": cells * args.steps / t_e2e / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": (La + Lb) * D * 4,
                "d2h_bytes_per_step": int(ph.shape[0]) * 8},
        "gpu_launches": kernels_per_wsdtw_step(args.nfrag, Lb) * args.steps,
        "clocks": clk.summary(),
    })
    al.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line only: skip the band, batch and bf16 blocks")
    ap.add_argument("--La", type=int, default=None,
                    help="override the pair's lengths (same recipe; for profiling smaller cases)")
    ap.add_argument("--Lb", type=int, default=None)
    ap.add_argument("--nfrag", type=int, default=32, help="WSDTW fragments (--config 5)")
    ap.add_argument("--config", type=int, default=1, choices=[1, 2, 3, 4, 5],
                    help="1: the 20000x25000 pair (default, the headline line); 2: the "
                         "256-pair batch; 3: the D = 128 pair with the BF16 cost; 4: the "
                         "100000x(100000-130000) pair in the learned band; 5: WSDTW of that "
                         "pair with --nfrag fragments")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.config == 2:
        run_batch(args)
    elif args.config == 3:
        run_precision(args)
    elif args.config == 4:
        run_band(args)
    elif args.config == 5:
        run_wsdtw(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
