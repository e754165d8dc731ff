"""Benchmark: proton histories/s of the Monte Carlo dose engine on one GB300.

Workload (one step): the heterogeneous slab phantom -- 128^3 voxels at 2 mm,
water / lung (-740 HU) / bone (+1200 HU) slabs of 20/40/10 mm -- with 400
spots on 10 energy layers (70-200 MeV, 5 mm grid, weights U[0.5,1.5]e6
protons) and 1e7 histories: history allocation, condensed-history transport
with the int64 tally, and normalisation to dose (all in the engine's
kernels).  ``value`` is histories/s with the grid resident in HBM; ``e2e`` is
the same metric through the C ABI with host buffers (grid and plan uploaded,
dose read back, every step).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own replica of the workload (histories are
independent, no collective on the data path) and rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "proton histories/s"
N_HIST = 10_000_000
SEED = 2
WORKLOAD = "slab phantom 128^3 at 2 mm (water/lung/bone), 400 spots on 10 layers 70-200 MeV, 1e7 histories"
# algorithmic thread-operations of one condensed-history step
OPS_PER_STEP = 230


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="engine", choices=["engine", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    p.add_argument("--histories", type=int, default=N_HIST,
                   help="histories per step (smaller cases for profiling; the metric's workload is 1e7)")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _workload():
    from paper_1809_03927_gb300 import workloads as W
    return W.slab_phantom(n=128), W.slab_plan(seed=SEED)


# ------------------------------------------------------------------ oracle
def _oracle_sample(phantom, plan, seconds_target=15.0):
    """The CPU oracle, as it stands, on a bounded sample of the workload:
    the first histories of the same 1e7-history run, all host cores."""
    import oracle
    oracle.build()
    n_probe = 2000
    t0 = time.perf_counter()
    oracle.transport(phantom, plan, N_HIST, SEED, hist_range=(0, n_probe))
    dt = time.perf_counter() - t0
    n = max(n_probe, min(int(n_probe * seconds_target / max(dt, 1e-3)), 2_000_000))
    t0 = time.perf_counter()
    r = oracle.transport(phantom, plan, N_HIST, SEED, hist_range=(n_probe, n_probe + n))
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": METRIC, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"histories [{n_probe}, {n_probe + n}) of the 1e7-history run ({n} histories, "
                      f"{dt:.1f} s, {r['steps'] / n:.1f} steps/history)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    phantom, plan = _workload()
    times, counts = [], []
    for i in range(args.warmup + args.steps):
        r = _oracle_sample(phantom, plan, seconds_target=4.0 if i < args.warmup else 10.0)
        if i >= args.warmup:
            n = float(r["sample"].split("(")[1].split(" ")[0])
            counts.append(n)
            times.append(n / r["value"])
    value = sum(counts) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * N_HIST / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{int(sum(counts))} histories over {args.steps} steps, each a bounded "
                                       "sample of the 1e7-history run; ms_per_step extrapolated"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ engine
def run_engine(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1809_03927_gb300 import dose as D

    phantom, plan = _workload()
    nx, ny, nz = phantom.n
    hu_host = np.ascontiguousarray(phantom.hu)
    spots = D.spots_array(plan)
    hu_dev = torch.from_numpy(hu_host).cuda()
    stream = torch.cuda.current_stream()
    ctx = D.dose_create_grid(nx, ny, nz, *phantom.d, phantom.origin, 1, hu_dev, phantom.beam_dir, stream)
    D.dose_add_spots(ctx, spots, None, stream)
    seed = SEED + 1000 * rank
    n_hist = args.histories
    # launch shape from the engine's autotuner (results do not depend on it)
    tune = D.dose_autotune(ctx, 0, n_hist, min(n_hist, 2_000_000), seed, stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        D.dose_run_phase(ctx, 0, n_hist, seed, 1.0, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()                       # evict L2 between steps (outside the timed events)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)

    # kernel-only time of the transport launch (dominant kernel), same stream
    kstart = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kend = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    jobs = D.make_jobs([dict(ctx=ctx, phase=0, n_histories=n_hist, seed=seed, flags=D.DOSE_JOB_CLEAR)])
    D.dose_run_batch(jobs, stream)
    jobs_run = D.make_jobs([dict(ctx=ctx, phase=0, n_histories=n_hist, seed=seed, flags=0)])
    torch.cuda.synchronize()
    tk = []
    for i in range(args.steps):
        flush.zero_()
        # clear without transport: a CLEAR job over an empty history range
        D.dose_run_batch(D.make_jobs([dict(ctx=ctx, phase=0, n_histories=n_hist, seed=seed,
                                           flags=D.DOSE_JOB_CLEAR, hist_begin=0, hist_end=0)]), stream)
        kstart[i].record(stream)
        D.dose_run_batch(jobs_run, stream)
        kend[i].record(stream)
    torch.cuda.synchronize()
    tk = [s.elapsed_time(e) for s, e in zip(kstart, kend)]
    clocks = sampler.stop()
    led = D.dose_read(ctx, D.DOSE_ENERGY_LEDGER, 0, np.zeros(8, np.uint64))
    steps_per_hist = float(led[4]) / float(led[5])

    # end to end through the C ABI with host buffers: upload grid + plan,
    # run, read the dose back to host memory, every step
    dose_host = torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory()
    hu_pinned = torch.from_numpy(hu_host).pin_memory()

    def e2e_step():
        c = D.dose_create_grid(nx, ny, nz, *phantom.d, phantom.origin, 1, hu_pinned, phantom.beam_dir, stream)
        try:
            D.dose_add_spots(c, spots, None, stream)
            D.dose_run_phase(c, 0, n_hist, seed, 1.0, None, stream)
            D.dose_read(c, D.DOSE_PHASE_DOSE, 0, dose_host, stream)
        finally:
            D.dose_destroy(c)

    e2e_s = float("nan")
    if not args.no_e2e:
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
    D.dose_destroy(ctx)

    # reduce over ranks: max time
    t_step = total_ms / args.steps
    vals = torch.tensor([t_step, e2e_s, sum(tk) / len(tk)], dtype=torch.float64, device="cuda")
    if ws > 1:
        torch.distributed.all_reduce(vals, op=torch.distributed.ReduceOp.MAX)
    t_step, e2e_s, t_kernel = [float(v) for v in vals.cpu()]
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    value = ws * n_hist / (t_step / 1e3)
    peaks = _peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_ops = sms * 128 * sm_mhz * 1e6 / 1e12          # Top/s: 128 FP32/INT32 lanes per SM
    achieved = n_hist * steps_per_hist * OPS_PER_STEP / (t_kernel / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (int64 tally, f64 normalisation)", "data": "synthetic",
        "config": {"workload": WORKLOAD if n_hist == N_HIST else WORKLOAD.replace("1e7", f"{n_hist:.0e}"),
                   "histories_per_step": n_hist, "steps_per_history": round(steps_per_hist, 2),
                   "l2": "256 MB buffer written between timed steps, outside the step events",
                   "launch": {"registers": "64" if tune[0] else "<=128", "block": tune[1], "chunk": tune[2],
                              "autotune_sample_us": tune[3]},
                   "parallelism": f"{ws} independent replica(s), one per GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Top/s",
                     "frac": achieved / peak_ops, "traffic": None,
                     "kernel": "k_transport", "kernel_ms": t_kernel,
                     "peak_basis": f"{sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (median sampled SM clock)",
                     "ops_per_step": OPS_PER_STEP},
        "e2e": {"value": ws * n_hist / e2e_s, "unit": METRIC,
                "h2d_bytes_per_step": int(hu_host.nbytes + len(plan) * 32),
                "d2h_bytes_per_step": int(nx * ny * nz * 4)},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _oracle_sample(phantom, plan)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_engine(args)


if __name__ == "__main__":
    main()
