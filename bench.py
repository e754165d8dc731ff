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
# Algorithmic work of one condensed-history step, in issue slots (thread
# operations): one Philox4x32-10 block (10 rounds of two 32x32->64 products
# and the key mixing), three Box-Muller transforms, about five table lerps,
# the voxel-face distances, the energy loss with its straggling, the
# scattering, frame and move, and one tally quantisation and atomic.  The
# estimate spans 300-450; this build's own narrower count is 230.  The
# headline fraction uses the low end, 300.
OPS_PER_STEP = 300
OPS_PER_STEP_RANGE = (230, 300, 450)
# DRAM bytes (read + write) of one transport launch on the slab workload
# (1e7 histories) per launch shape it was measured in (registers variant,
# block, chunk, material grid), from ncu --metrics dram__bytes_read.sum,
# dram__bytes_write.sum on the full-size launch of the current kernel
# (bench.py --launch R,B,C,M; the single-job kernel with subnormals flushed,
# built for all physics on and the launch's material source).
TRANSPORT_DRAM = {(1, 1024, 32, 1): 3.81e6, (1, 1024, 64, 1): 3.47e6, (1, 1024, 128, 1): 3.83e6,
                  (1, 1024, 256, 1): 3.47e6, (1, 1024, 64, 0): 2.74e6, (1, 1024, 128, 0): 2.74e6}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="engine", choices=["engine", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    p.add_argument("--no-4d", action="store_true", help="skip the 4D-plan measurement")
    p.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    p.add_argument("--no-ragged", action="store_true", help="skip the ragged-batch measurement")
    p.add_argument("--no-trials", action="store_true", help="skip the uncertainty-trials measurement")
    p.add_argument("--histories-trial", type=int, default=4_000_000,
                   help="histories per phase of each uncertainty trial")
    p.add_argument("--serve-window", type=float, default=5.0, help="seconds of Poisson arrivals")
    p.add_argument("--serve-rate", type=float, default=20.0, help="mean arrivals per second")
    p.add_argument("--serve-policies", default="fair,shortest_first",
                   help="server sharing policies to measure: fair (equal shares), shortest_first, "
                        "shortest_first_bounded (with --serve-max-wait)")
    p.add_argument("--serve-max-wait", type=int, default=8,
                   help="max_wait_steps of the shortest_first_bounded policy")
    p.add_argument("--serve-budget-gb", type=float, default=150.0, help="device memory for request slots")
    p.add_argument("--serve-low-rate", type=float, default=8.0,
                   help="mean arrivals per second of the second serving point (below capacity)")
    p.add_argument("--serve-low-window", type=float, default=30.0,
                   help="seconds of arrivals of the second serving point (0: skip it)")
    p.add_argument("--histories-4d", type=int, default=100_000_000, help="histories per phase of the 4D plan")
    p.add_argument("--small-4d", action="store_true",
                   help="4D leg on a 128x128x80 grid at 2x2x5 mm (profiler captures), not the 4DCT workload")
    p.add_argument("--reference-seconds", type=float, default=5.0,
                   help="CPU seconds of each timed oracle step of the reference arm")
    p.add_argument("--launch", default=None,
                   help="transport launch shape 'registers,block,chunk,material' instead of the autotuner's")
    p.add_argument("--histories", type=int, default=N_HIST,
                   help="histories per step (smaller cases for profiling; the metric's workload is 1e7)")
    return p.parse_args()


def reduce_max_over_ranks(values, ws, device="cpu"):
    """Per-rank times -> the maximum over the ranks (all ranks get it); the
    process group (nccl for the engine, any backend in tests) is already
    initialised when ws > 1."""
    import torch
    vals = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    return [float(v) for v in vals.cpu()]


def job_throughput(ws, units_per_rank, step_ms):
    """Whole-job throughput: the units every rank processed in one step over
    the slowest rank's step time (weak scaling: each rank has its own)."""
    return ws * units_per_rank / (step_ms / 1e3)


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
def _interleaved(phantom, plan, seconds_target, nthreads=None):
    """The oracle on every stride-th history of the 1e7-history run (h mod
    stride == 0, so the sample has the run's mix of spots and energies),
    the stride chosen from two probes (a fixed cost plus a cost per history)
    so the sample takes about seconds_target.  Returns (histories/s,
    histories, seconds, steps/history, stride)."""
    import oracle

    def run(stride):
        t0 = time.perf_counter()
        r = oracle.transport(phantom, plan, N_HIST, SEED, batch=(0, stride), nthreads=nthreads)
        return time.perf_counter() - t0, r

    (t1, r1), (t2, r2) = run(5000), run(1000)
    per = max((t2 - t1) / max(r2["histories"] - r1["histories"], 1), 1e-9)
    stride = max(1, min(1000, int(N_HIST * per / seconds_target)))
    dt, r = run(stride)
    return r["histories"] / dt, r["histories"], dt, r["steps"] / r["histories"], stride


def _oracle_sample(phantom, plan, seconds_target=15.0):
    """The CPU oracle, as it stands, on a bounded sample of the workload:
    every stride-th history of the same 1e7-history run, all host cores."""
    import oracle
    oracle.build()
    rate, n, dt, sph, stride = _interleaved(phantom, plan, seconds_target)
    return {"value": rate, "unit": METRIC, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"every {stride}th history of the 1e7-history run ({n} histories, {dt:.1f} s, "
                      f"{sph:.1f} steps/history, the run's 91.8)"}


def _oracle_extra(phantom, plan):
    """More oracle figures for the CPU baseline: one thread on the same
    interleaved sample, the single-pencil workload run in full, and the 4D
    plan extrapolated from samples."""
    import oracle
    from paper_1809_03927_gb300 import workloads as W
    out = {}
    rate, n, dt, sph, stride = _interleaved(phantom, plan, 5.0, nthreads=1)
    out["one_thread"] = {"value": rate, "unit": METRIC, "cores": 1,
                         "sample": f"every {stride}th history ({n} histories, {dt:.1f} s)"}
    wph, wpl = W.water_phantom(), W.pencil_plan(150.0, 4.0)
    t0 = time.perf_counter()
    oracle.transport(wph, wpl, 100_000, 1)
    dt = time.perf_counter() - t0
    out["pencil_full"] = {"value": 100_000 / dt, "unit": METRIC, "seconds": dt, "cores": os.cpu_count(),
                          "workload": "150 MeV pencil, sigma 4 mm, water 64x64x160 at 2 mm, 1e5 histories, in full"}
    # 4D plan: the timeline in full, every phase's transport from a sample of
    # its subplan, the EMTM from one phase on a slab of the grid; scaled to
    # 10 phases x 1e8 histories and the whole grid (extrapolated)
    ph, dvf, geo = W.phantom_4dct()
    plan4 = W.tumour_plan(geo, ph.origin)
    dl = W.Delivery(seed=3)
    t0 = time.perf_counter()
    pp, _, _ = oracle.timeline(plan4, dl)
    t_tl = time.perf_counter() - t0
    busiest = int(np.argmax(pp.sum(axis=1)))
    n_s = 20_000
    t0 = time.perf_counter()
    oracle.transport(ph, plan4.with_protons(pp[busiest]), 100_000_000, SEED, phase=busiest, stream=busiest,
                     batch=(0, 100_000_000 // n_s))
    t_per_hist = (time.perf_counter() - t0) / n_s
    n_ph = int(np.count_nonzero(pp.sum(axis=1)))
    z0, z1 = 70, 78                                     # 8 of 160 slices, one source phase
    rho = np.stack([oracle.density(ph, p)[z0:z1] for p in (0, 1)]).astype(np.float32)
    dose = np.ones((2,) + rho.shape[1:], np.float32)
    t0 = time.perf_counter()
    oracle.emtm(dose, rho, ph.d, 0, (2, 2, 5), dvf=np.ascontiguousarray(dvf[:2, :, z0:z1]))
    t_emtm = (time.perf_counter() - t0) * (ph.n[2] / (z1 - z0)) * (ph.n_phases - 1)
    s_plan = t_tl + n_ph * 100_000_000 * t_per_hist + t_emtm
    out["four_d_extrapolated"] = {
        "s_per_plan": s_plan, "extrapolated": True, "timeline_s": t_tl,
        "transport_s_per_history": t_per_hist, "phases": n_ph, "emtm_s": t_emtm, "cores": os.cpu_count(),
        "sample": f"timeline in full; {n_s} histories of phase {busiest} (all cores) scaled to {n_ph} phases x 1e8; "
                  f"EMTM of one source phase on {z1 - z0} of {ph.n[2]} slices (one thread) scaled to 9 phases x "
                  "the whole grid"}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    phantom, plan = _workload()
    times, counts = [], []
    for i in range(args.warmup + args.steps):
        r = _oracle_sample(phantom, plan, seconds_target=min(4.0, args.reference_seconds) if i < args.warmup
                           else args.reference_seconds)
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


# ------------------------------------------------------------------ 4D plan
def _bench_4d(D, torch, stream, n_per_phase, reps, seed, small=False):
    """Seconds per 4D dose of the synthetic 4DCT: 10 phases of 256x256x160
    at 1x1x2.5 mm, 3000 spots on 20 layers (70-180 MeV), delivery timeline
    (1e9 p/s, 2 ms spot switch, 1 s layer switch, 4 s period, random start),
    n_per_phase histories per phase in one launch, EMTM accumulation onto
    phase 0 with 2x2x5 subvoxels (0.5 mm) and the Eq. 2 sum.  Grids, DVFs
    and plan are resident; the timed plan runs the timeline, all phases'
    transport and the accumulation.  small: the same phantom on a 128x128x80
    grid at 2x2x5 mm (for profiler captures of the accumulation kernels)."""
    from paper_1809_03927_gb300 import workloads as W
    ph, dvf, geo = W.phantom_4dct(128, 128, 80, (2.0, 2.0, 5.0)) if small else W.phantom_4dct()
    plan = W.tumour_plan(geo, ph.origin)
    dlv = D.delivery_struct(W.Delivery(seed=3))
    nx, ny, nz = ph.n
    hu_dev = torch.from_numpy(np.ascontiguousarray(ph.hu)).cuda()
    dvf_dev = torch.from_numpy(dvf).cuda()
    pull_dev = torch.from_numpy(W.reference_to_phase_field(dvf)).cuda()
    # the registrations as a DIR system would store them: each phase's
    # field on a grid of every other CT voxel centre (2 x 2 x 5 mm)
    reg_grid = dict(n=(nx // 2, ny // 2, nz // 2), start_mm=tuple(ph.origin[k] + 0.5 * ph.d[k] for k in range(3)),
                    spacing_mm=tuple(2.0 * v for v in ph.d), row_cos=(1, 0, 0), col_cos=(0, 1, 0))
    reg_delta = [torch.from_numpy(np.ascontiguousarray(np.moveaxis(dvf[p][:, ::2, ::2, ::2], 0, -1))).cuda()
                 for p in range(ph.n_phases)]
    del dvf
    ctx = D.dose_create_grid(nx, ny, nz, *ph.d, ph.origin, ph.n_phases, hu_dev, ph.beam_dir, stream)
    spots = D.spots_array(plan)
    try:
        D.dose_add_spots(ctx, spots, dlv, stream)
        phase_p = D.dose_read(ctx, D.DOSE_SUBPLAN, 0, np.zeros((ph.n_phases, len(plan)), np.uint64)).sum(axis=1)
        tune = D.dose_autotune(ctx, int(np.argmax(phase_p)), n_per_phase, min(n_per_phase, 10_000_000), seed, stream)
        material = D.dose_get_option(ctx, D.DOSE_OPT_MATERIAL_GRID)

        def plan_once():
            D.dose_add_spots(ctx, spots, dlv, stream)
            D.dose_run_4d(ctx, n_per_phase, seed, 0, (2, 2, 5), dvf=dvf_dev, stream=stream)

        plan_once()
        torch.cuda.synchronize()
        walls, evs = [], []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            plan_once()
            e1.record(stream)
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - t0)
            evs.append(e0.elapsed_time(e1) / 1e3)
        acc_batched = D.dose_read(ctx, D.DOSE_ACCUM, 0, np.zeros((nz, ny, nx), np.float32))

        # the plain engine: the same plan and histories, one phase job per
        # launch (each phase's allocation, transport and normalisation), then
        # the same accumulation; phase doses and the accumulated dose are the
        # same bits as the batched plan's (histories are keyed by seed,
        # history and phase)
        zero = torch.zeros(nx * ny * nz, dtype=torch.float32, device="cuda")

        def plan_plain():
            D.dose_add_spots(ctx, spots, dlv, stream)
            for p in range(ph.n_phases):
                if phase_p[p] > 0:
                    D.dose_run_phase(ctx, p, n_per_phase, seed, 1.0, None, stream)
                else:
                    D.dose_set_phase_dose(ctx, p, zero, stream)
            D.dose_accumulate_subvoxel(ctx, 0, (2, 2, 5), dvf=dvf_dev, stream=stream)

        plain_walls = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan_plain()
            torch.cuda.synchronize()
            plain_walls.append(time.perf_counter() - t0)
        plain_same = bool(np.array_equal(D.dose_read(ctx, D.DOSE_ACCUM, 0, np.zeros((nz, ny, nx), np.float32)),
                                         acc_batched))
        del zero
        # the accumulation alone
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        D.dose_accumulate_subvoxel(ctx, 0, (2, 2, 5), dvf=dvf_dev, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        emtm_s = e0.elapsed_time(e1) / 1e3
        stats = D.dose_read(ctx, D.DOSE_EMTM_STATS, 0, np.zeros(4, np.uint64))
        # both accumulation methods against the subvoxel count (the paper's
        # study of n): EMTM pushes with the phase->reference field, DIM
        # pulls with the reference->phase field
        study = {}
        for name, method, field in (("emtm", D.ACCUM_EMTM, dvf_dev), ("dim", D.ACCUM_DIM, pull_dev)):
            study[name] = {}
            for nsub in ((1, 1, 1), (2, 2, 2), (2, 2, 5), (4, 4, 4)):
                ts = []
                for _ in range(2):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    D.dose_accumulate_subvoxel(ctx, 0, nsub, dvf=field, method=method, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1) / 1e3)
                study[name]["x".join(map(str, nsub))] = min(ts)
        # decoding every phase's registration onto the CT grid (App. B)
        nvox = nx * ny * nz
        decoded = torch.empty(ph.n_phases * 3 * nvox, dtype=torch.float32, device="cuda")
        dmask = torch.empty(nvox, dtype=torch.uint8, device="cuda")
        ts = []
        for _ in range(3):
            dmask.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for p in range(1, ph.n_phases):
                D.dose_decode_dvf(ctx, reg_grid, reg_delta[p], decoded[p * 3 * nvox:(p + 1) * 3 * nvox],
                                  mask=dmask, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        decode_s = min(ts)
        del decoded, dmask
        steps = sum(int(D.dose_read(ctx, D.DOSE_ENERGY_LEDGER, p, np.zeros(8, np.uint64))[4])
                    for p in range(ph.n_phases) if phase_p[p] > 0)
        n_run = int(np.count_nonzero(phase_p)) * n_per_phase
    finally:
        D.dose_destroy(ctx)
    s_plan = float(np.median(walls))
    return {"s_per_plan": s_plan, "s_per_plan_device": float(np.median(evs)), "reps": reps,
            "plain_s_per_plan": float(np.median(plain_walls)), "plain_same_dose": plain_same,
            "histories_per_plan": n_run, "histories_per_s": n_run / s_plan,
            "steps_per_history": steps / n_run, "emtm_s": emtm_s,
            "emtm_subvoxels": int(stats[0]), "emtm_atomic_pairs": int(stats[2]),
            "dim_s": study["dim"]["2x2x5"], "accumulation_s_by_subvoxels": study,
            "dvf_decode_s": decode_s,
            "dvf_decode": f"{ph.n_phases - 1} registrations on {nx // 2}x{ny // 2}x{nz // 2} grids "
                          "(every other CT voxel centre) decoded onto the CT grid with the report mask",
            "workload": ("synthetic 4DCT 10 x 128x128x80 at 2x2x5 mm (small, for profiling)" if small else
                         "synthetic 4DCT 10 x 256x256x160 at 1x1x2.5 mm") + ", 3000 spots / 20 layers 70-180 MeV, "
                        f"{n_per_phase:.0e} histories per phase, EMTM 2x2x5 onto phase 0",
            "launch": {"registers": "64" if tune[0] else "<=128", "block": tune[1], "chunk": tune[2],
                       "material_grid": material}}


# ------------------------------------------------------------------ uncertainty trials
def _bench_trials(D, torch, stream, n_per_phase, n_trials=25, seed=SEED):
    """The uncertainty study of Sec. 2.B on the synthetic 4DCT: 25 trials,
    each drawing its start phase (random), breathing period (3-7 s, whole
    seconds) and synchrotron parameters (App. A fill model: 1.25e10 protons
    (2 nC) per fill, 8 s extraction limit, 70 ms discard, 2 s reset, 2 ms
    spot switch, 1e9 p/s, each with a Gaussian spread) as one launch of the
    timeline, then every trial's phase subplans transported in ONE ragged
    persistent launch (n_per_phase histories per phase with protons), then
    each trial's EMTM onto phase 0.  Reported: seconds for the whole study
    and the transport's histories/s."""
    from paper_1809_03927_gb300 import workloads as W
    ph, dvf, geo = W.phantom_4dct()
    plan = W.tumour_plan(geo, ph.origin)
    nx, ny, nz = ph.n
    S_ = 1_000_000_000
    mean = W.Delivery(seed=seed, start_phase=-1, synchrotron=1, fill_protons=12_500_000_000,
                      extraction_limit_ns=8 * S_, discard_ns=70_000_000, layer_switch_ns=2 * S_,
                      spot_switch_ns=2_000_000, rate_protons_per_s=1_000_000_000)
    spread = W.DeliverySpread(period_min_ns=3 * S_, period_max_ns=7 * S_, period_step_ns=S_,
                              spot_switch_sigma_ns=200_000, layer_switch_sigma_ns=100_000_000,
                              discard_sigma_ns=5_000_000, rate_sigma=50_000_000,
                              fill_protons_sigma=500_000_000, extraction_limit_sigma_ns=300_000_000)
    hu_dev = torch.from_numpy(np.ascontiguousarray(ph.hu)).cuda()
    dvf_dev = torch.from_numpy(dvf).cuda()
    del dvf
    base = D.dose_create_grid(nx, ny, nz, *ph.d, ph.origin, ph.n_phases, hu_dev, ph.beam_dir, stream)
    views = []
    spots = D.spots_array(plan)
    try:
        views = [D.dose_create_view(base) for _ in range(n_trials)]

        def study():
            D.dose_add_spots_trials(views, spots, D.delivery_struct(mean), D.spread_struct(spread), 0, stream)
            jobs = []
            for k, v in enumerate(views):
                pp = D.dose_read(v, D.DOSE_SUBPLAN, 0, np.zeros((ph.n_phases, len(plan)), np.uint64))
                for p in range(ph.n_phases):
                    if pp[p].sum():
                        jobs.append(dict(ctx=v, phase=p, n_histories=n_per_phase, seed=seed + k))
                    else:
                        D.dose_set_phase_dose(v, p, torch.zeros(nx * ny * nz, dtype=torch.float32, device="cuda"),
                                              stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            D.dose_run_batch(D.make_jobs(jobs), stream)
            e1.record(stream)
            for v in views:
                D.dose_accumulate_subvoxel(v, 0, (2, 2, 5), dvf=dvf_dev, stream=stream)
            torch.cuda.synchronize()
            return len(jobs), e0.elapsed_time(e1) / 1e3

        D.dose_add_spots_trials(views, spots, D.delivery_struct(mean), D.spread_struct(spread), 0, stream)
        # launch shape of the study's batch, tuned on a 2e7-history sample of it
        tjobs = []
        for k, v in enumerate(views):
            pp = D.dose_read(v, D.DOSE_SUBPLAN, 0, np.zeros((ph.n_phases, len(plan)), np.uint64))
            tjobs += [dict(ctx=v, phase=p, n_histories=n_per_phase, seed=seed + k)
                      for p in range(ph.n_phases) if pp[p].sum()]
        tune = D.dose_autotune_batch(D.make_jobs(tjobs), 20_000_000, stream)
        study()                                    # warm-up (and first allocation of the views)
        t0 = time.perf_counter()
        n_jobs, mc_s = study()
        wall = time.perf_counter() - t0
        periods = sorted({int(D.read_delivery(v)["period_ns"]) // S_ for v in views})
        acc = [D.dose_read(v, D.DOSE_ACCUM, 0, np.zeros((nz, ny, nx), np.float32)) for v in views[:3]]
        steps = 0
        for v in views:
            pp = D.dose_read(v, D.DOSE_SUBPLAN, 0, np.zeros((ph.n_phases, len(plan)), np.uint64)).sum(axis=1)
            steps += sum(int(D.dose_read(v, D.DOSE_ENERGY_LEDGER, p, np.zeros(8, np.uint64))[4])
                         for p in range(ph.n_phases) if pp[p] > 0)

        # the plain engine: the same trials, one dose_run_phase per phase
        # job, then the same accumulations; the same bits as the batch
        zero = torch.zeros(nx * ny * nz, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D.dose_add_spots_trials(views, spots, D.delivery_struct(mean), D.spread_struct(spread), 0, stream)
        for k, v in enumerate(views):
            pp = D.dose_read(v, D.DOSE_SUBPLAN, 0, np.zeros((ph.n_phases, len(plan)), np.uint64))
            for p in range(ph.n_phases):
                if pp[p].sum():
                    D.dose_run_phase(v, p, n_per_phase, seed + k, 1.0, None, stream)
                else:
                    D.dose_set_phase_dose(v, p, zero, stream)
        for v in views:
            D.dose_accumulate_subvoxel(v, 0, (2, 2, 5), dvf=dvf_dev, stream=stream)
        torch.cuda.synchronize()
        plain_wall = time.perf_counter() - t0
        plain_same = all(np.array_equal(D.dose_read(v, D.DOSE_ACCUM, 0, np.zeros((nz, ny, nx), np.float32)), a)
                         for v, a in zip(views[:3], acc))
    finally:
        for v in views:
            D.dose_destroy(v)
        D.dose_destroy(base)
    return {"s_per_study": wall, "trials": n_trials, "phase_jobs": n_jobs, "transport_s": mc_s,
            "plain_s_per_study": plain_wall, "plain_same_dose": plain_same,
            "launch": {"registers": "64" if tune[0] else "<=128", "block": tune[1], "chunk": tune[2]},
            "transport_histories_per_s": n_jobs * n_per_phase / mc_s, "periods_s_drawn": periods,
            "steps_per_history": steps / (n_jobs * n_per_phase),
            # the transport launch against the measured issue peak at the
            # headline 300 issue slots per step
            "transport_steps_per_s": steps / mc_s,
            "workload": f"{n_trials} uncertainty trials of the synthetic 4DCT plan (synchrotron fills, "
                        f"period U{{3..7}} s, Gaussian machine parameters), {n_per_phase:.0e} histories per "
                        "phase with protons, all trials' phases in one ragged launch, EMTM 2x2x5 per trial"}


# ------------------------------------------------------------------ ragged batch
def _bench_ragged(D, torch, stream, n_random=62, seed=4, reps=2):
    """A ragged batch of dose jobs in one persistent launch against the plain
    engine (one job per launch): 62 random cube phantoms (64-256 voxels a
    side at 2 mm, random slabs and spheres), 20-5000 spots (70-220 MeV), 1e5-5e7
    histories (log-uniform), plus the 4DCT plan delivered with 4x layer
    repainting and with 30 %-duty gating (phases 4-6), every phase it reaches
    a job of its own (1e7 histories each)."""
    from paper_1809_03927_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    ctxs, specs = [], []
    try:
        for _ in range(n_random):
            side = int(rng.choice(np.arange(64, 257, 16)))
            ph = W.random_phantom(rng, side)
            pl = W.random_plan(rng, W.log_uniform_int(rng, 20, 5000), side * 2.0 * 0.3)
            n = W.log_uniform_int(rng, 1e5, 5e7)
            c = D.dose_create_grid(side, side, side, *ph.d, ph.origin, 1,
                                   torch.from_numpy(np.ascontiguousarray(ph.hu)).cuda(), ph.beam_dir, stream)
            ctxs.append(c)
            D.dose_add_spots(c, D.spots_array(pl), None, stream)
            specs.append(dict(ctx=c, phase=0, n_histories=n, seed=int(rng.integers(1, 2 ** 62))))
        ph4, _, geo = W.phantom_4dct(with_dvf=False)
        plan4 = W.tumour_plan(geo, ph4.origin)
        hu4 = torch.from_numpy(np.ascontiguousarray(ph4.hu)).cuda()
        for dl in (W.Delivery(seed=3, repaints=4), W.Delivery(seed=3, gated=1, gate_first=4, gate_last=6)):
            c = D.dose_create_grid(*ph4.n, *ph4.d, ph4.origin, ph4.n_phases, hu4, ph4.beam_dir, stream)
            ctxs.append(c)
            D.dose_add_spots(c, D.spots_array(plan4), D.delivery_struct(dl), stream)
            pp = D.dose_read(c, D.DOSE_SUBPLAN, 0, np.zeros((ph4.n_phases, len(plan4)), np.uint64)).sum(axis=1)
            for p in range(ph4.n_phases):
                if pp[p] > 0:
                    specs.append(dict(ctx=c, phase=p, n_histories=10_000_000, seed=77 + p))
        total = sum(sp["n_histories"] for sp in specs)
        jobs = D.make_jobs(specs)
        # the batch's launch shape from the batch autotuner (a 2e7-history
        # sample spread over the jobs), set on every context
        tune = D.dose_autotune_batch(jobs, 20_000_000, stream)
        D.dose_run_batch(jobs, stream)                    # warm-up
        torch.cuda.synchronize()
        tb = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            D.dose_run_batch(jobs, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            tb.append(e0.elapsed_time(e1) / 1e3)
        # one job per launch: the single-job shape, tuned on the largest job
        big = max(specs, key=lambda sp: sp["n_histories"])
        tune1 = D.dose_autotune(big["ctx"], big["phase"], big["n_histories"], 2_000_000, 1, stream)
        for c in ctxs:
            for opt, v in ((D.DOSE_OPT_REGISTERS, tune1[0]), (D.DOSE_OPT_BLOCK, tune1[1]), (D.DOSE_OPT_CHUNK, tune1[2])):
                D.dose_set_option(c, opt, v)
        for sp in specs:                                  # warm-up
            D.dose_run_phase(sp["ctx"], sp["phase"], sp["n_histories"], sp["seed"], 1.0, None, stream)
        torch.cuda.synchronize()
        tp = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for sp in specs:
                D.dose_run_phase(sp["ctx"], sp["phase"], sp["n_histories"], sp["seed"], 1.0, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            tp.append(e0.elapsed_time(e1) / 1e3)
    finally:
        for c in ctxs:
            D.dose_destroy(c)
    return {"jobs": len(specs), "histories": total, "batched_s": float(np.median(tb)),
            "batched_histories_per_s": total / float(np.median(tb)), "plain_s": float(np.median(tp)),
            "plain_histories_per_s": total / float(np.median(tp)),
            "launch": {"registers": "64" if tune[0] else "<=128", "block": tune[1], "chunk": tune[2]},
            "plain_launch": {"registers": "64" if tune1[0] else "<=128", "block": tune1[1], "chunk": tune1[2]}}


# ------------------------------------------------------------------ serving
def _requests(window_s, rate, seed=5):
    """Poisson arrivals (seeded exponential gaps) of robust-scenario requests:
    nominal, +-3 mm setup shift on one axis, or +-3.5 % stopping-power scale;
    total histories log-uniform in [1e6, 1e8] (split over the phases)."""
    rng = np.random.default_rng(seed)
    scen = [(1.0, (0.0, 0.0, 0.0))]
    for ax in range(3):
        for sgn in (1.0, -1.0):
            sh = [0.0, 0.0, 0.0]
            sh[ax] = 3.0 * sgn
            scen.append((1.0, tuple(sh)))
    scen += [(1.035, (0.0, 0.0, 0.0)), (0.965, (0.0, 0.0, 0.0))]
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > window_s:
            return out
        spr, sh = scen[int(rng.integers(len(scen)))]
        n = int(round(float(np.exp(rng.uniform(np.log(1e6), np.log(1e8))))))
        out.append(dict(t=t, n=n, seed=int(rng.integers(1, 2 ** 62)), spr=spr, shift=sh))


def _serve_schedule(D, base, spots, dlv, dvf_dev, budget_bytes, reqs, stream, hist, policy, max_wait=0):
    """Replay the arrival schedule through a server with the given sharing
    policy; latency percentiles, throughput and where the makespan went."""
    srv = D.dose_server_create(base, budget_bytes, 40_000_000, spots, dlv, min_slice=20_000,
                               nsub=(2, 2, 5), dvf=dvf_dev, policy=policy, max_wait_steps=max_wait)
    done_at, k, t0, ids, max_active = {}, 0, time.perf_counter(), {}, 0
    window_s = reqs[-1]["t"] if reqs else 0.0
    at_window_end = None                      # requests in the system when the last one arrives
    try:
        while len(done_at) < len(reqs):
            now = time.perf_counter() - t0
            while k < len(reqs) and reqs[k]["t"] <= now:
                r = reqs[k]
                ids[D.dose_server_submit(srv, r["n"], r["seed"], r["spr"], r["shift"])] = k
                k += 1
            st = D.dose_server_stats(srv)
            max_active = max(max_active, st["active"] + st["queued"])
            if at_window_end is None and k == len(reqs):
                at_window_end = st["active"] + st["queued"]
            if st["queued"] + st["active"] == 0:
                time.sleep(max(0.0, min(0.005, reqs[k]["t"] - now)) if k < len(reqs) else 0.0)
                continue
            for rid in D.dose_server_step(srv, stream):
                done_at[ids[rid]] = time.perf_counter() - t0
                D.dose_server_release(srv, rid)
        total_s = time.perf_counter() - t0
        st = D.dose_server_stats(srv)
        tm = D.dose_server_timing(srv)
    finally:
        D.dose_server_destroy(srv)
    lat = [done_at[i] - reqs[i]["t"] for i in range(len(reqs))]
    busy = tm["step_wall_s"]
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(np.mean(lat)), "histories_per_s": hist / total_s, "makespan_s": total_s,
            "steps": st["steps"], "slots": st["slots"], "max_in_system": max_active,
            "in_system_at_last_arrival": at_window_end,
            "slot_gb": st["slot_bytes"] / 1e9,
            # where the makespan went: steps (device batch, device
            # accumulation, host remainder of the step) and idle time
            # waiting for arrivals
            "breakdown_s": {"transport_batches": tm["batch_s"], "accumulations": tm["accumulate_s"],
                            "host_step_overhead": max(busy - tm["batch_s"] - tm["accumulate_s"], 0.0),
                            "idle_between_steps": max(total_s - busy, 0.0)},
            "histories_per_device_batch_s": hist / tm["batch_s"] if tm["batch_s"] > 0 else None}


def _bench_serving(D, torch, stream, window_s, rate, budget_bytes, policies, max_wait=8):
    """p50/p99 latency (arrival -> dose ready) and histories/s of the
    continuous-batching server against the plain engine (each request alone,
    one phase job per launch, first come first served) on the same arrival
    schedule over the resident 4DCT."""
    from paper_1809_03927_gb300 import workloads as W
    ph, dvf, geo = W.phantom_4dct()
    plan = W.tumour_plan(geo, ph.origin)
    dlv = D.delivery_struct(W.Delivery(seed=3))
    spots = D.spots_array(plan)
    nx, ny, nz = ph.n
    hu_dev = torch.from_numpy(np.ascontiguousarray(ph.hu)).cuda()
    dvf_dev = torch.from_numpy(dvf).cuda()
    del dvf
    reqs = _requests(window_s, rate)
    base = D.dose_create_grid(nx, ny, nz, *ph.d, ph.origin, ph.n_phases, hu_dev, ph.beam_dir, stream)
    out = {"requests": len(reqs), "window_s": window_s, "rate_per_s": rate,
           "offered_histories_per_s": sum(r["n"] for r in reqs) / window_s}
    try:
        # launch shapes from the autotuners: the server's steps are batches of
        # several requests (tuned on two requests' phases in one batch; the
        # slots take the base's options), the plain engine runs one phase
        # job per launch (tuned on the fullest phase)
        probe = D.dose_create_view(base)
        D.dose_add_spots(probe, spots, dlv, stream)
        pp = D.dose_read(probe, D.DOSE_SUBPLAN, 0, np.zeros((ph.n_phases, len(plan)), np.uint64)).sum(axis=1)
        phases = [p for p in range(ph.n_phases) if pp[p] > 0]
        probe2 = D.dose_create_view(base)
        D.dose_add_spots(probe2, spots, dlv, stream)
        tune = D.dose_autotune_batch(D.make_jobs([dict(ctx=v, phase=p, n_histories=5_000_000, seed=1 + k)
                                                  for k, v in enumerate((probe, probe2)) for p in phases]),
                                     20_000_000, stream)
        mat = D.dose_get_option(probe2, D.DOSE_OPT_MATERIAL_GRID)
        D.dose_destroy(probe2)
        for opt, v in ((D.DOSE_OPT_REGISTERS, tune[0]), (D.DOSE_OPT_BLOCK, tune[1]), (D.DOSE_OPT_CHUNK, tune[2]),
                       (D.DOSE_OPT_MATERIAL_GRID, mat)):
            D.dose_set_option(base, opt, v)
        tune1 = D.dose_autotune(probe, int(np.argmax(pp)), 10_000_000, 2_000_000, 1, stream)

        # ---- served: continuous batching, under each sharing policy
        hist = sum(r["n"] // len(phases) * len(phases) for r in reqs)
        for key, policy, wait in (("served", D.DOSE_SERVE_FAIR, 0),
                                  ("served_shortest_first", D.DOSE_SERVE_SHORTEST_FIRST, 0),
                                  ("served_shortest_first_bounded", D.DOSE_SERVE_SHORTEST_FIRST, max_wait)):
            if key in policies:
                out[key] = _serve_schedule(D, base, spots, dlv, dvf_dev, budget_bytes, reqs, stream, hist, policy,
                                           wait)
                out[key]["policy"] = policies[key]
                if wait:
                    out[key]["max_wait_steps"] = wait

        # capacity: the served rate while the device is busy (histories per
        # second of transport batches); an offered load above it grows the
        # queue, which the records show as requests in the system when the
        # last request arrives
        rates = [out[k]["histories_per_device_batch_s"]
                 for k in ("served", "served_shortest_first", "served_shortest_first_bounded")
                 if k in out and out[k]["histories_per_device_batch_s"]]
        if rates:
            out["capacity_histories_per_s"] = max(rates)
            out["offered_over_capacity"] = out["offered_histories_per_s"] / max(rates)
            out["above_capacity"] = out["offered_over_capacity"] > 1.0

        # ---- plain: one request at a time, one phase job per launch
        done_at, t0, k = {}, time.perf_counter(), 0
        for i, r in enumerate(reqs):
            now = time.perf_counter() - t0
            if r["t"] > now:
                time.sleep(r["t"] - now)
            n_pp = max(1, r["n"] // len(phases))
            for p in range(ph.n_phases):
                if p in phases:
                    D.dose_run_phase(probe, p, n_pp, r["seed"], r["spr"], r["shift"], stream)
            D.dose_accumulate_subvoxel(probe, 0, (2, 2, 5), dvf=dvf_dev, stream=stream)
            torch.cuda.current_stream().synchronize()
            done_at[i] = time.perf_counter() - t0
        total_s = time.perf_counter() - t0
        D.dose_destroy(probe)
        lat = [done_at[i] - reqs[i]["t"] for i in range(len(reqs))]
        out["plain"] = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                        "mean_s": float(np.mean(lat)), "histories_per_s": hist / total_s, "makespan_s": total_s}
        out["launch"] = {"registers": "64" if tune[0] else "<=128", "block": tune[1], "chunk": tune[2]}
        out["plain_launch"] = {"registers": "64" if tune1[0] else "<=128", "block": tune1[1], "chunk": tune1[2]}
    finally:
        D.dose_destroy(base)
    return out


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
    # launch shape from the engine's autotuner, timed on the whole run (before
    # the timed region; results do not depend on the shape), or as given
    if args.launch:
        regs, block, chunk, mat = (int(v) for v in args.launch.split(","))
        for opt, v in ((D.DOSE_OPT_REGISTERS, regs), (D.DOSE_OPT_BLOCK, block), (D.DOSE_OPT_CHUNK, chunk),
                       (D.DOSE_OPT_MATERIAL_GRID, mat)):
            D.dose_set_option(ctx, opt, v)
        tune = (regs, block, chunk, 0)
    else:
        tune = D.dose_autotune(ctx, 0, n_hist, n_hist, seed, stream)
    # the device's measured issue and atomic peaks (a few ms, before the timed region)
    measured = D.dose_measure_peaks(stream)
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
    launch_opts = {o: D.dose_get_option(ctx, o) for o in (D.DOSE_OPT_REGISTERS, D.DOSE_OPT_BLOCK, D.DOSE_OPT_CHUNK,
                                                         D.DOSE_OPT_MATERIAL_GRID)}
    dose_host = torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory()
    hu_pinned = torch.from_numpy(hu_host).pin_memory()

    def e2e_step():
        c = D.dose_create_grid(nx, ny, nz, *phantom.d, phantom.origin, 1, hu_pinned, phantom.beam_dir, stream)
        try:
            # the launch shape tuned once above, as a user would reuse it
            for opt, v in launch_opts.items():
                D.dose_set_option(c, opt, v)
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
    material = D.dose_get_option(ctx, D.DOSE_OPT_MATERIAL_GRID)
    D.dose_destroy(ctx)

    # whole-job time: the slowest rank
    t_step, e2e_s, t_kernel = reduce_max_over_ranks([total_ms / args.steps, e2e_s, sum(tk) / len(tk)], ws,
                                                    device="cuda")
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    value = job_throughput(ws, n_hist, t_step)
    peaks = _peaks()
    shape = (int(tune[0]), int(tune[1]), int(tune[2]), material)
    # DRAM traffic of the transport launch, from an ncu capture of this
    # workload in this launch shape (null for any other shape or size)
    traffic = TRANSPORT_DRAM.get(shape) if n_hist == N_HIST else None
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    nominal = sms * 128 * sm_mhz * 1e6 / 1e12          # Top/s: 128 FP32/INT32 lanes per SM
    peak_ops = measured["issue_mixed"] / 1e12
    steps_per_s = n_hist * steps_per_hist / (t_kernel / 1e3)
    achieved = steps_per_s * OPS_PER_STEP / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (int64 tally, f64 normalisation)", "data": "synthetic",
        "config": {"workload": WORKLOAD if n_hist == N_HIST else WORKLOAD.replace("1e7", f"{n_hist:.0e}"),
                   "histories_per_step": n_hist, "steps_per_history": round(steps_per_hist, 2),
                   "l2": "256 MB buffer written between timed steps, outside the step events",
                   "launch": {"registers": "64" if tune[0] else "<=128", "block": tune[1], "chunk": tune[2],
                              "material_grid": material, "autotune_sample_us": tune[3]},
                   "parallelism": f"{ws} independent replica(s), one per GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Top/s",
                     "frac": achieved / peak_ops, "traffic": traffic,
                     # the single-job kernel built for all physics on and
                     # the material source in use (<7, 1>: grid, <7, 2>: HU)
                     "kernel": ("k_transport1_r64" if tune[0] else "k_transport1") + ("<7, 1>" if material else "<7, 2>"),
                     "kernel_ms": t_kernel,
                     "ops_per_step": OPS_PER_STEP,
                     "frac_by_ops_per_step": {str(k): steps_per_s * k / 1e12 / peak_ops for k in OPS_PER_STEP_RANGE},
                     "peak_basis": f"measured: mixed FP32/INT32 instruction stream (dose_measure_peaks), "
                                   f"{peak_ops:.2f} Top/s; nominal {sms} SMs x 128 lanes x {sm_mhz:.0f} MHz = "
                                   f"{nominal:.2f} Top/s; FFMA alone {measured['issue_ffma'] / 1e12:.2f} Top/s",
                     # the bound in histories/s: the slower of issue (300 slots per
                     # step) and the tally atomics (one per step), per history
                     "histories_per_s_bound": min(measured["issue_mixed"] / (steps_per_hist * OPS_PER_STEP),
                                                  measured["atomic_u64"] / steps_per_hist),
                     "histories_per_s_kernel": n_hist / (t_kernel / 1e3),
                     "atomic": {"achieved": steps_per_s, "peak": measured["atomic_u64"], "unit": "atomics/s",
                                "frac": steps_per_s / measured["atomic_u64"],
                                "basis": "one 64-bit tally atomic per step against measured u64 atomic additions "
                                         "to random elements of a 16.8 MB L2-resident array"}},
        "e2e": {"value": ws * n_hist / e2e_s, "unit": METRIC,
                "h2d_bytes_per_step": int(hu_host.nbytes + len(plan) * 32),
                "d2h_bytes_per_step": int(nx * ny * nz * 4)},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if not args.no_4d:
        line["four_d"] = _bench_4d(D, torch, stream, args.histories_4d, 2, SEED, small=args.small_4d)
    if not args.no_ragged:
        line["ragged_batch"] = _bench_ragged(D, torch, stream)
    if not args.no_trials:
        line["uncertainty_trials"] = _bench_trials(D, torch, stream, args.histories_trial)
    if not args.no_serve:
        pol = {"fair": "served", "shortest_first": "served_shortest_first",
               "shortest_first_bounded": "served_shortest_first_bounded"}
        policies = {pol[v.strip()]: v.strip() for v in args.serve_policies.split(",") if v.strip()}
        line["serving"] = _bench_serving(D, torch, stream, args.serve_window, args.serve_rate,
                                         int(args.serve_budget_gb * 1e9), policies, args.serve_max_wait)
        if args.serve_low_window > 0:
            line["serving_below_capacity"] = _bench_serving(D, torch, stream, args.serve_low_window,
                                                            args.serve_low_rate, int(args.serve_budget_gb * 1e9),
                                                            policies, args.serve_max_wait)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _oracle_sample(phantom, plan)
        line["cpu_baseline"].update(_oracle_extra(phantom, plan))
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
