"""Benchmark of the transport hot path on one GB300 (particle-steps per second).

Workload (one "step" of this benchmark = one pass of the whole hot path):
  1 degree global grid 360 x 181 x 60 levels (log-spaced 1000 -> 10 hPa), wind =
  seeded sum of 64 Fourier modes on the sphere (20 m/s rms u, v; 0.5 Pa/s rms
  omega), 4 snapshots 6 h apart (24 h periodic); 1e6 particles uniform in
  lon/lat/ln p; dt = 180 s over 24 h = 480 fused steps of advection + turbulent
  (Dx = 50, Dz = 0.1 m^2/s) + mesoscale diffusion (Philox normals), particles
  sorted by met cell every 20 steps; 5 snapshot loads (repack) per pass.
  Each pass restarts from the same initial particle state.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line.
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

DT = 180.0
DT_MET = 21600.0
T_END = 86400.0
N_PART = 1_000_000
SORT_EVERY = 20
SEED_FIELD = 2
SEED_PART = 2
SEED_RNG = 2
# DRAM bytes (read + write) of one fused-step launch of this workload by
# (particle groups, particles per thread) -- a launch covers 1/groups of the
# particles -- from ncu captures of full-size launches of variant 2 with the
# hand-off to the sort (see profiles/).  A schedule without a capture reports
# None, and so does any launch after the kernel changes, until it is captured again.
TRAFFIC_PER_LAUNCH = {(2, 1): 156314880,   # 142.14 MB read + 14.18 MB written, 5e5 particles
                      (2, 2): 157370112,   # 142.99 + 14.38 MB
                      (2, 4): 157224704}   # 143.92 + 13.30 MB
# sha256 (first 16 hex digits) of the fused step's sources when the counters
# were taken; a different hash means the kernel changed and traffic is None
TRAFFIC_KERNEL_SHA = "e3d7de66b08ecba8"
TRAFFIC_SOURCES = ("paper_2211_12616_gb300/csrc/step.cu", "paper_2211_12616_gb300/csrc/internal.h",
                   "paper_2211_12616_gb300/csrc/cell_key.cuh", "paper_2211_12616_gb300/csrc/met_record.cuh")


def kernel_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]
METRIC = "particle-steps/s on 1 GB300 (advect+diffuse) and % gather roofline, surrogate vs plain"
WORKLOAD = ("1deg 360x181x60 Fourier-mode wind, 4 snapshots 6h apart, 1e6 particles, dt=180s, 24h "
            "(480 fused advect+turb+meso steps), sort by met cell every 20 steps")


def _config(n, extra=None):
    c = {"workload": WORKLOAD, "grid": "360x181x60", "particles": n, "steps_per_pass": int(T_END / DT),
         "dt_s": DT, "sort_every": SORT_EVERY, "met_storage": "fp32",
         "l2": "inputs larger than L2 (~0.45 GB of met sources, slots, particles and sort workspace per pass)"}
    if extra:
        c.update(extra)
    return c


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# Algorithmic operations of one fused step of one particle (advection +
# turbulent + mesoscale diffusion), counted from the method's formulas, not from
# the kernel: one operation per add, multiply, fused multiply-add, compare,
# conversion or integer op.  The position update counts as the method states it
# (three float64 additions), not as the float-float arithmetic that stands in for
# them; the Philox key schedule is per seed, not per particle-step.  The kernel
# executes more instructions (addressing, predication, clamps, float-float).
ALU_OPS_PER_PARTICLE_STEP = {
    "locate, 2 evaluations x (lon 5 + lat 5 + level search 6)": 32,
    "trilinear, 2 evaluations x 2 snapshots x 3 variables x 7 lerps x 2 + time lerps 2 x 3 x 2": 180,
    "subgrid variance: corner weights 12 + 2 snapshots x 3 variables x 8 corners x 3 + time lerps 6": 162,
    "midpoint stages: 3 increments x 3, twice; midpoint position rules 6": 24,
    "Philox4x32-10, 2 calls x 10 rounds x (2 wide multiplies = 4 + 4 xor)": 160,
    "Box-Muller, 3 pairs x (2 uniforms x 2 + -2 ln u 1 + angle 1 + 2 products)": 24,
    "turbulent + mesoscale displacements and AR(1) update": 34,
    "position update: increments summed 3 x 2, then 3 float64 additions": 9,
    "position rules": 6,
}
ALU_OPS = sum(ALU_OPS_PER_PARTICLE_STEP.values())
# transcendentals, charged against the special-function units' own rate
MUFU_OPS_PER_PARTICLE_STEP = {
    "cos(lat): midpoint stage 1, stage 2, diffusion conversion": 3,
    "Box-Muller, 3 pairs x (log, sqrt, sin, cos)": 12,
}
MUFU_OPS = sum(MUFU_OPS_PER_PARTICLE_STEP.values())
MUFU_PER_SM_PER_CLK = 16      # 4 results per clock on each of the SM's 4 sub-partitions
# per-step stencil gather of the gather roofline: 2 evaluations x 8 corners x one
# 32-byte pair record (a corner's u, v, omega, T on both snapshots, float32)
L2_BYTES_PER_PARTICLE_STEP = 2 * 8 * 32
# particle stream of one launch, per particle: lon, lat, p (float64) and u', v', w'
# (float32) read and written, id and release id read
PARTICLE_STREAM_BYTES = 2 * (3 * 8 + 3 * 4) + 2 * 4


def measure_copy_gbs(dev, mb, reps):
    """Bandwidth of mptrac_copy_probe on two buffers of ``mb`` MiB: read + write bytes of one launch
    of ``reps`` repetitions (loads and stores cached in L2 only) over its CUDA-event time, the best
    of 5 launches after 2 warm-up launches.  Changes no setting of the GPU."""
    import torch

    import paper_2211_12616_gb300 as M
    n = mb * (1 << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    best = 0.0
    for i in range(7):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        M.copy_probe(a, b, reps)
        e1.record()
        torch.cuda.synchronize()
        if i >= 2:
            best = max(best, 2 * 4 * n * reps / (e0.elapsed_time(e1) / 1000.0) / 1e9)
    del a, b
    return best


def measure_l2_gbs(dev):
    """L2 bandwidth: the copy probe on source and destination of 8, 16 and 24 MiB each (resident in
    L2 together), 100 repetitions per launch; the best size."""
    return max(measure_copy_gbs(dev, mb, 100) for mb in (8, 16, 24))


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def great_circle_km(lon1, lat1, lon2, lat2):
    """Haversine distance on the sphere of radius 6371 km (degrees in)."""
    p1, p2 = np.radians(lat1), np.radians(lat2)
    dl = np.radians(np.asarray(lon2) - np.asarray(lon1))
    h = np.sin((p2 - p1) / 2) ** 2 + np.cos(p1) * np.cos(p2) * np.sin(dl / 2) ** 2
    return 2 * 6371.0 * np.arcsin(np.sqrt(np.clip(h, 0.0, 1.0)))


def final_subset(parts, n_sub):
    """lon, lat, p of the particles with id < n_sub, in id order."""
    d = parts.to_numpy()
    keep = d["id"] < n_sub
    o = np.argsort(d["id"][keep])
    return {k: d[k][keep][o] for k in ("lon", "lat", "p")}


def error_summary(got, ref):
    km = great_circle_km(got["lon"], got["lat"], ref["lon"], ref["lat"])
    dp = np.abs(got["p"] - ref["p"]) / ref["p"]
    return {"km_median": float(np.median(km)), "km_p99": float(np.quantile(km, 0.99)), "km_max": float(km.max()),
            "dp_rel_median": float(np.median(dp)), "dp_rel_p99": float(np.quantile(dp, 0.99))}


# launch schedule of the batched form in the default line (the autotuner's choice on this
# workload: register corner cache with 128 registers, one sort per met interval)
BATCH_SCHEDULE = {"variant": 1, "persistent": False, "per_thread": 1, "sort_every": 120}


def storage_figures(dev, grid, snaps, init, best, steps, warmup, n_sub, fp32_ms):
    """The headline workload with the met fields stored as bf16 or fp16 with level scales:
    rate, speed-up over float32 storage, and the final positions of the first particles."""
    import torch

    import paper_2211_12616_gb300 as M
    from paper_2211_12616_gb300.simulation import Simulation, periodic_snapshots

    out, finals = {}, {}
    stream = torch.cuda.Stream(device=dev)
    for name, storage in (("bf16", M.MPTRAC_BF16), ("fp16", M.MPTRAC_FP16)):
        ctx = M.Context(grid, storage)
        ctx.set_launch(best["variant"], best["persistent"], best.get("per_thread", 1))
        work = init.clone()
        sim = Simulation(ctx, periodic_snapshots(snaps, DT_MET), DT_MET, work, DT, M.DiffParams(), SEED_RNG,
                         SORT_EVERY, groups=best["groups"])

        def one_pass():
            with torch.cuda.stream(stream):
                work.copy_(init)
                sim.run(0.0, T_END, stream=stream)
        for _ in range(warmup):
            one_pass()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            one_pass()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out[name] = {"ms_per_pass": ms, "particle_steps_per_s": init.n * (T_END / DT) / (ms / 1000.0),
                     "speedup_vs_fp32": fp32_ms / ms, "slot_bytes": int(grid.npoints * 8)}
        finals[name] = final_subset(work, n_sub)
        ctx.close()
        del sim, work
    return out, finals


# --------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# --------------------------------------------------------------------------
def _oracle_setup(offset: int, n: int):
    from oracle import transport as tr
    from oracle.driver import run_schedule
    from workloads import fourier_modes, fourier_snapshot, grid_1deg_60lev, uniform_particles
    grid = grid_1deg_60lev()
    modes = fourier_modes(SEED_FIELD)
    snaps = [fourier_snapshot(grid, modes, h * DT_MET) for h in range(4)]
    st = uniform_particles(N_PART, grid.plev, SEED_PART)
    sub = {k: v[offset:offset + n] for k, v in st.items()}
    at = lambda t: snaps[int(round(t / DT_MET)) % 4]
    return lambda t_end: run_schedule(grid, at, DT_MET, sub, 0.0, t_end, DT, tr.DiffParams(), SEED_RNG)


def oracle_sample_rate(n_sample: int, t_end: float = T_END):
    """Times the FP64 oracle on the first ``n_sample`` particles of the workload (this process);
    returns (particle-steps/s, seconds, the oracle's final state of those particles)."""
    run = _oracle_setup(0, n_sample)
    t0 = time.perf_counter()
    final = run(t_end)
    el = time.perf_counter() - t0
    psteps = n_sample * (t_end / DT)
    return psteps / el, el, final


def _oracle_worker(offset, n, t_end, barrier, out):
    run = _oracle_setup(offset, n)
    barrier.wait()
    t0 = time.perf_counter()
    run(t_end)
    out.put(time.perf_counter() - t0)


def oracle_all_cores(n_per: int, workers: int, t_end: float = T_END):
    """The oracle on ``workers`` host processes at once (spawned: this process may hold a CUDA
    context), each on its own ``n_per`` particles of the workload; returns (particle-steps/s of
    all of them, seconds of the slowest).  The oracle itself is unchanged: particles are
    independent, so the processes share nothing."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(workers), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(q * n_per, n_per, t_end, barrier, out)) for q in range(workers)]
    for pr in procs:
        pr.start()
    els = [out.get() for _ in procs]
    for pr in procs:
        pr.join()
    el = max(els)
    return workers * n_per * (t_end / DT) / el, el


def run_reference(args, rank, world):
    if rank != 0:
        return
    n_per = int(os.environ.get("BENCH_ORACLE_SAMPLE", "2000"))
    workers = os.cpu_count() or 1
    times = []
    for i in range(args.warmup + args.steps):
        _, el = oracle_all_cores(n_per, workers)
        if i >= args.warmup:
            times.append(el)
    n_sample = n_per * workers
    value = len(times) * n_sample * (T_END / DT) / sum(times)
    sample = (f"{workers} processes x {n_per} particles of the workload (disjoint), full 24 h (480 steps) per "
              f"step, numpy float64 on every host core")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(args.particles, {"oracle_sample_particles": n_sample}),
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": workers, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist

    import paper_2211_12616_gb300 as M
    from paper_2211_12616_gb300.simulation import Simulation, periodic_snapshots
    from workloads import fourier_modes, fourier_snapshot, grid_1deg_60lev, uniform_particles

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    n = args.particles
    grid = grid_1deg_60lev()
    modes = fourier_modes(SEED_FIELD)
    snaps = [fourier_snapshot(grid, modes, h * DT_MET, device=dev, as_numpy=False) for h in range(4)]
    from paper_2211_12616_gb300.replicas import aggregate_rate, id_offset, max_over_ranks
    st0 = uniform_particles(n, grid.plev, SEED_PART + 1000 * rank, id0=id_offset(rank, n))
    init = M.Particles.from_numpy(st0, device=dev)
    work = init.clone()
    ctx = M.Context(grid, {"fp32": M.MPTRAC_FP32, "bf16": M.MPTRAC_BF16, "fp16": M.MPTRAC_FP16}[args.storage])
    prm = M.DiffParams()
    stream = torch.cuda.Stream(device=dev)
    sims = {}

    def sim_for(groups):
        if groups not in sims:
            sims[groups] = Simulation(ctx, periodic_snapshots(snaps, DT_MET), DT_MET, work, DT, prm, SEED_RNG,
                                      SORT_EVERY, groups=groups)
        return sims[groups]
    psteps_per_pass = n * int(round(T_END / DT))

    # timing of the dominant kernel (the fused step): CUDA events around every launch on
    # the stream it is launched on; with several particle groups the launches of different
    # groups overlap, so the kernel's busy time is the union of the launch intervals
    ev_pairs = []

    def hook(stage, s):
        e = torch.cuda.Event(enable_timing=True)
        e.record(s)
        if stage == "begin":
            ev_pairs.append([e, None, s])
        else:
            for pair in reversed(ev_pairs):
                if pair[2] is s and pair[1] is None:
                    pair[1] = e
                    break

    # launch schedule picked by the autotuner on one met interval of this workload
    from paper_2211_12616_gb300.autotune import autotune, candidates

    def make(cfg):
        sim_c = sim_for(cfg["groups"])

        def go():
            ctx.set_launch(cfg["variant"], cfg["persistent"], cfg["per_thread"])
            with torch.cuda.stream(stream):
                sim_c.run(0.0, 2 * DT_MET, stream=stream)   # two intervals: one overlapped met load
        return go

    groups_try = (args.groups,) if args.groups else (1, 2, 3)
    if args.variant >= 0:   # fixed schedule (profiling): no autotuner launches before the timed pass
        best = {"variant": args.variant, "persistent": False, "per_thread": args.per_thread, "sort_every": SORT_EVERY,
                "groups": args.groups or 2}
        tune_ms = {}
    else:
        best, tune_ms = autotune(make, lambda: work.copy_(init),
                                 candidates(sort_every=(SORT_EVERY,), groups=groups_try), stream, repeats=3)
    ctx.set_launch(best["variant"], best["persistent"], best["per_thread"])
    sim = sim_for(best["groups"])

    def one_pass():
        with torch.cuda.stream(stream):
            work.copy_(init)
            sim.run(0.0, T_END, stream=stream)

    for _ in range(args.warmup):
        one_pass()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    sim.step_hook = hook
    l0 = M.load().mptrac_kernel_launches()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(args.steps):
        one_pass()
    end.record(stream)
    torch.cuda.synchronize()
    launches = M.load().mptrac_kernel_launches() - l0
    sim.step_hook = None
    ms = start.elapsed_time(end)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms)
    value = aggregate_rate(psteps_per_pass * args.steps, world, ms_max)
    # launch intervals relative to the start event; their union is the kernel's busy time
    iv = sorted((start.elapsed_time(a), start.elapsed_time(b)) for a, b, _ in ev_pairs)
    busy, cur0, cur1 = 0.0, None, None
    for a0, a1 in iv:
        if cur1 is None or a0 > cur1:
            if cur1 is not None:
                busy += cur1 - cur0
            cur0, cur1 = a0, a1
        else:
            cur1 = max(cur1, a1)
    if cur1 is not None:
        busy += cur1 - cur0
    step_ms = [a.elapsed_time(b) for a, b, _ in ev_pairs]
    n_groups = best["groups"]
    # per launch: the particles of one group over SORT_EVERY steps; busy time per launch
    # counts overlapping launches of different groups once
    psteps_per_launch = n * SORT_EVERY / n_groups
    step_avg_ms = busy / len(step_ms)

    # ---- end-to-end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        host_init = {k: getattr(init, k).cpu().pin_memory() for k in M.Particles.FIELDS if getattr(init, k) is not None}
        host_snaps = [{k: v.cpu().pin_memory() for k, v in s.items()} for s in snaps]
        out_host = {k: torch.empty(n, dtype=torch.float64).pin_memory() for k in ("lon", "lat", "p")}
        sim_h = Simulation(ctx, periodic_snapshots(host_snaps, DT_MET), DT_MET, work, DT, prm, SEED_RNG, SORT_EVERY,
                           groups=best["groups"])
        h2d = sum(t.numel() * t.element_size() for t in host_init.values())
        h2d += 5 * sum(t.numel() * t.element_size() for t in host_snaps[0].values())
        d2h = sum(t.numel() * t.element_size() for t in out_host.values())

        def e2e_pass():
            with torch.cuda.stream(stream):
                for k, v in host_init.items():
                    getattr(work, k).copy_(v, non_blocking=True)
                sim_h.run(0.0, T_END, stream=stream)
                for k, v in out_host.items():
                    v.copy_(getattr(work, k), non_blocking=True)
        for _ in range(max(1, args.warmup // 2)):
            e2e_pass()
        torch.cuda.synchronize()
        s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s2.record(stream)
        k2 = max(1, args.steps)
        for _ in range(k2):
            e2e_pass()
        e2.record(stream)
        torch.cuda.synchronize()
        ms2 = max_over_ranks(s2.elapsed_time(e2))
        e2e = {"value": aggregate_rate(psteps_per_pass * k2, world, ms2), "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "copies": "particle state in and final lon/lat/p out: torch copies between pinned host buffers "
                         "and the device on the timed stream; the 5 met snapshots: mptrac_load_met from pinned "
                         "host memory (prefetched on a copy stream by the Simulation); compute through the C ABI"}

    # ---- the added forms on the same GPU: 16-bit storage, batched releases, surrogate ----
    forms, finals = None, {}
    n_sub = int(os.environ.get("BENCH_ORACLE_SAMPLE", "8000"))
    if world == 1 and not args.no_forms and args.storage == "fp32":   # the forms compare against fp32 storage
        finals["fp32"] = final_subset(work, n_sub)
        t_forms = time.perf_counter()
        storage, f16 = storage_figures(dev, grid, snaps, init, best, max(1, args.steps // 2), 1, n_sub,
                                       ms_max / args.steps)
        finals.update(f16)
        forms = {"storage": storage,
                 "batch": batch_figures(dev, grid, snaps, 2, 1, schedule=BATCH_SCHEDULE),
                 "surrogate": surrogate_figures(dev, grid, snaps, 10_000_000, 10_000_000, 4)}
        forms["seconds"] = time.perf_counter() - t_forms
        torch.cuda.empty_cache()

    if rank != 0:
        return
    hbm_peak, peak_kind = _peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_max_mhz") or 2070.0
    kernel_rate = psteps_per_launch / (step_avg_ms / 1000.0)       # particle-steps/s of the step launches
    alu_peak = n_sm * 128 * sm_mhz * 1e6 / 1e12          # TOP/s: one op per lane per clock
    alu_achieved = ALU_OPS * kernel_rate / 1e12
    mufu_peak = n_sm * MUFU_PER_SM_PER_CLK * sm_mhz * 1e6 / 1e12
    mufu_achieved = MUFU_OPS * kernel_rate / 1e12
    # the gather roofline: T = max(B_HBM / BW_HBM, B_L2 / BW_L2) per particle-step, with
    # B_L2 the per-step stencil gather and B_HBM the particle stream plus the compulsory met
    # bytes (every pair record of the interval read once per launch: an upper bound)
    l2_gbs = measure_l2_gbs(dev)
    stream_b = PARTICLE_STREAM_BYTES * (n / n_groups) / psteps_per_launch
    rec_b = 32.0 if args.storage == "fp32" else 16.0        # bytes of a pair record
    met_b = rec_b * grid.nx * grid.ny * grid.nz / psteps_per_launch
    b_hbm = stream_b + met_b
    b_l2 = L2_BYTES_PER_PARTICLE_STEP * rec_b / 32.0
    t_roof = max(b_hbm / (hbm_peak * 1e9), b_l2 / (l2_gbs * 1e9))
    traffic = (TRAFFIC_PER_LAUNCH.get((n_groups, best["per_thread"]))
               if best["variant"] == 2 and not best["persistent"] and kernel_sha() == TRAFFIC_KERNEL_SHA
               and args.storage == "fp32" else None)
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": _config(n, {"autotuned": best, "autotune_ms": tune_ms,
                                                   "met_storage": args.storage}),
        "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TOP/s",
                     "frac": alu_achieved / alu_peak,
                     "traffic": traffic,
                     "kernel_sha": kernel_sha(),
                     "kernel": "k_transport<fp32, step>", "avg_launch_ms": step_avg_ms,
                     "launches_timed": len(step_ms), "particle_steps_per_launch": psteps_per_launch,
                     "timing": "union of the launch intervals (CUDA events on each group's stream) / launches",
                     "mean_event_ms_per_launch": sum(step_ms) / len(step_ms),
                     "ops_per_particle_step": ALU_OPS,
                     "ops_counted": "the method's operations (bench.py ALU_OPS_PER_PARTICLE_STEP), not the kernel's",
                     "peak_kind": f"derived: {n_sm} SMs x 128 lanes x {sm_mhz:.0f} MHz, one op per lane per clock",
                     "mufu": {"ops_per_particle_step": MUFU_OPS, "achieved": mufu_achieved, "peak": mufu_peak,
                              "unit": "TOP/s", "frac": mufu_achieved / mufu_peak,
                              "peak_kind": f"derived: {n_sm} SMs x {MUFU_PER_SM_PER_CLK} per clock x "
                                           f"{sm_mhz:.0f} MHz"}},
        "gather_roofline": {"b_l2_per_particle_step": b_l2, "l2_gbs": l2_gbs,
                            "l2_kind": "measured here: device copy resident in L2 (read + write bytes)",
                            "b_hbm_per_particle_step": b_hbm, "hbm_gbs": hbm_peak,
                            "hbm_kind": f"{peak_kind} hbm_gbs",
                            "t_roof_ns": t_roof * 1e9, "roofline_particle_steps_per_s": 1.0 / t_roof,
                            "achieved_particle_steps_per_s": kernel_rate,
                            "frac": kernel_rate * t_roof,
                            "pass_frac": value * t_roof,
                            "hbm_only_particle_steps_per_s": hbm_peak * 1e9 / b_hbm,
                            "hbm": ({"traffic_bytes_per_launch": traffic,
                                     "achieved_gbs": traffic / (step_avg_ms / 1000.0) / 1e9,
                                     "frac": traffic / (step_avg_ms / 1000.0) / 1e9 / hbm_peak}
                                    if traffic else None),
                            "note": "the per-step stencil gather term assumes no reuse between steps; the kernel "
                                    "keeps a cell's corners in registers while the particle stays in the cell, "
                                    "so it is bound by the ALU roofline, and the HBM-only bound is given beside"},
        "clocks": clk, "gpu_launches": int(launches),
        "e2e": e2e,
        "forms": forms,
    }
    if not args.no_cpu_baseline:
        n_sample = int(os.environ.get("BENCH_ORACLE_SAMPLE", "8000"))
        workers = os.cpu_count() or 1
        rate1, el1, oracle_final = oracle_sample_rate(n_sample)
        rate, el = oracle_all_cores(n_sample // 2, workers)
        line["cpu_baseline"] = {"value": rate, "unit": "particle-steps/s", "cores": workers, "kind": "oracle",
                                "sample": f"{workers} processes x {n_sample // 2} particles of the 1e6 (disjoint), "
                                          f"full 24 h (480 steps), {el:.1f} s of numpy float64 on every host core",
                                "single_core": {"value": rate1, "sample": f"first {n_sample} particles, "
                                                f"full 24 h, {el1:.1f} s on one core"}}
        # the oracle's final state of the same particles is the reference of the storage forms
        if forms is not None and n_sample == n_sub:
            for name, fin in finals.items():
                err = error_summary(fin, oracle_final)
                if name == "fp32":
                    line["accuracy_vs_oracle"] = dict(err, particles=n_sub)
                else:
                    forms["storage"][name].update(err)
    print(json.dumps(line), flush=True)
    ctx.close()


# --------------------------------------------------------------------------
# batched releases (64 column releases, 72 h, CUDA graphs, autotuned schedule)
# --------------------------------------------------------------------------
BATCH_RELEASES, BATCH_SEED, BATCH_T_END = 64, 4, 72 * 3600.0


def batch_figures(dev, grid, snaps, steps, warmup, count_scale=1.0, schedule=None):
    """Batched releases on one GPU: rate of the 72 h pass replayed from CUDA graphs.

    ``schedule`` None: the autotuner picks the launch variant, persistence and sort interval
    on one met interval; else that schedule (dict variant, persistent, per_thread, sort_every)."""
    import torch

    import paper_2211_12616_gb300 as M
    from paper_2211_12616_gb300.autotune import autotune, candidates
    from paper_2211_12616_gb300.batch import BatchedRun
    from paper_2211_12616_gb300.simulation import periodic_snapshots
    from workloads import column_releases

    rel = column_releases(BATCH_RELEASES, BATCH_SEED, count_scale=count_scale)
    init = M.Particles.from_numpy(rel.particles, device=dev)
    work = init.clone()
    ctx = M.Context(grid, M.MPTRAC_FP32)
    prm = M.DiffParams()
    stream = torch.cuda.Stream(device=dev)
    at = periodic_snapshots(snaps, DT_MET)
    # active particle-steps of one 72 h pass: steps n with n dt in [0, t_end) of each release
    n_steps_total = int(round(BATCH_T_END / DT))
    steps_active = np.minimum(np.ceil(rel.t_end / DT), n_steps_total)
    psteps = float((rel.counts * steps_active).sum())

    def sched(cfg):   # the schedule keys BatchedRun takes (one particle group: graphs span all releases)
        return {k: cfg[k] for k in ("variant", "persistent", "per_thread", "sort_every")}

    if schedule is None:
        def make(cfg):
            run = BatchedRun(ctx, at, DT_MET, work, rel.t_start, rel.t_end, DT, prm, SEED_RNG, **sched(cfg))
            return lambda: run.run_eager(0.0, DT_MET, stream=stream)
        best, timings = autotune(make, lambda: work.copy_(init), candidates(), stream, repeats=1)
    else:
        best, timings = dict(schedule), None
    run = BatchedRun(ctx, at, DT_MET, work, rel.t_start, rel.t_end, DT, prm, SEED_RNG, **sched(best))
    work.copy_(init)
    run.run_eager(0.0, DT_MET, stream=stream)      # first-use set-up outside capture
    torch.cuda.synchronize()
    run.capture(0.0, BATCH_T_END, stream)

    def one_pass():
        with torch.cuda.stream(stream):
            work.copy_(init)
            run.replay()

    for _ in range(warmup):
        one_pass()
    torch.cuda.synchronize()
    l0 = M.load().mptrac_kernel_launches()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        one_pass()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    out = {"particle_steps_per_s": psteps / (ms / 1000.0), "ms_per_pass": ms, "particles": int(rel.counts.sum()),
           "active_particle_steps_per_pass": psteps, "schedule": best, "autotuned": schedule is None,
           "candidates_ms": timings, "host_launches_in_timed_region": int(M.load().mptrac_kernel_launches() - l0),
           "workload": f"{BATCH_RELEASES} column releases (1-20 km), counts log-uniform 1e3-1e6 x {count_scale}, "
                       "durations 6-72 h, 1deg 60-level field, 72 h, CUDA graph per met interval"}
    run = None
    ctx.close()
    return out


def run_batch(args, rank, world):
    import torch

    from workloads import fourier_modes, fourier_snapshot, grid_1deg_60lev

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    grid = grid_1deg_60lev()
    modes = fourier_modes(SEED_FIELD)
    snaps = [fourier_snapshot(grid, modes, h * DT_MET, device=dev, as_numpy=False) for h in range(4)]
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    f = batch_figures(dev, grid, snaps, args.steps, args.warmup, args.count_scale)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": f["particle_steps_per_s"], "unit": "particle-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": f["ms_per_pass"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f["workload"] + ", autotuned schedule", "particles": f["particles"],
                       "active_particle_steps_per_pass": f["active_particle_steps_per_pass"],
                       "autotuned": f["schedule"], "candidates_ms": f["candidates_ms"]},
            "clocks": clk, "gpu_launches_captured": "graph replay (launch counter counts host launches only)",
            "host_launches_in_timed_region": f["host_launches_in_timed_region"]}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# precision: 0.3 degree x 137 levels, u/v/omega/T in fp32 / bf16 / fp16 storage
# --------------------------------------------------------------------------
PREC_T_END, PREC_SEED, PREC_N, PREC_SUB = 12 * 3600.0, 3, 10_000_000, 10_000


PREC_HORIZONS = (3600.0, 21600.0, 43200.0)


def _precision_subset_gpu(M, grid, snaps, storage, sub, diffuse):
    """The subset stepped alone (its trajectories do not depend on other particles) on this
    storage: states at every horizon, and u, v, omega, T sampled at the 12 h positions."""
    import torch
    ctx = M.Context(grid, storage, nvars=4)
    for slot in (0, 1):
        f = snaps[slot]
        ctx.load_met(slot, slot * DT_MET, f["u"], f["v"], f["w"], f["T"])
    parts = M.Particles.from_numpy(sub)
    prm = M.DiffParams(turb=diffuse, meso=diffuse)
    out, step, t = {}, 0, 0.0
    for h in PREC_HORIZONS:
        while t < h:
            if t >= 2 * DT_MET - 1e-6:
                raise ValueError("horizon beyond the loaded snapshots")
            if t >= DT_MET - 1e-6 and step == int(round(DT_MET / DT)):
                f = snaps[2]
                ctx.load_met(2, 2 * DT_MET, f["u"], f["v"], f["w"], f["T"])
            t_next = min(h, (math.floor(t / DT_MET + 1e-9) + 1) * DT_MET)
            n_steps = int(round((t_next - t) / DT))
            ctx.step(parts, t, DT, prm, SEED_RNG, step, n_steps)
            step += n_steps
            t = t_next
        torch.cuda.synchronize()
        d = parts.to_numpy()
        o = np.argsort(d["id"])
        out[h] = {k: d[k][o] for k in ("lon", "lat", "p")}
    sampled = ctx.sample_met(parts, PREC_HORIZONS[-1]).cpu().numpy()[:, np.argsort(parts.to_numpy()["id"])]
    ctx.close()
    return out, sampled


def _precision_oracle(grid, host, sub, diffuse):
    """The float64 oracle on the subset: states at every horizon (the cpu_baseline leg)."""
    from oracle import transport as tr
    prm = tr.DiffParams(turb=diffuse, meso=diffuse)
    mets = [tr.Met(grid, q * DT_MET, {k: host[q][k] for k in ("u", "v", "w")},
                   (q + 1) * DT_MET, {k: host[q + 1][k] for k in ("u", "v", "w")}) for q in (0, 1)]
    out, st, step, t = {}, sub, 0, 0.0
    for h in PREC_HORIZONS:
        while t < h:
            q = int(math.floor(t / DT_MET + 1e-9))
            t_next = min(h, (q + 1) * DT_MET)
            n_steps = int(round((t_next - t) / DT))
            st = tr.step(mets[q], st, t, DT, prm, SEED_RNG, step, n_steps)
            step += n_steps
            t = t_next
        out[h] = {k: st[k] for k in ("lon", "lat", "p")}
    return out


def run_precision(args, rank, world):
    import torch

    import paper_2211_12616_gb300 as M
    from paper_2211_12616_gb300.simulation import Simulation
    from workloads import fourier_modes, fourier_snapshot, grid_03deg_137lev, uniform_particles

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    grid = grid_03deg_137lev()
    modes = fourier_modes(PREC_SEED, n_modes=256, multiscale=True, with_T=True)
    snaps = [fourier_snapshot(grid, modes, h * DT_MET, device=dev, as_numpy=False) for h in range(3)]
    n = args.particles if args.particles != N_PART else PREC_N
    st0 = uniform_particles(n, grid.plev, PREC_SEED)
    init = M.Particles.from_numpy(st0, device=dev)
    prm = M.DiffParams()
    stream = torch.cuda.Stream(device=dev)
    sub_ids = np.linspace(0, n - 1, min(PREC_SUB, n)).astype(np.int64)
    sub = {k: v[sub_ids] for k, v in st0.items()}
    psteps = n * int(round(PREC_T_END / DT))
    at = lambda t: (snaps[int(round(t / DT_MET))]["u"], snaps[int(round(t / DT_MET))]["v"],
                    snaps[int(round(t / DT_MET))]["w"], snaps[int(round(t / DT_MET))]["T"])
    results, subset = {}, {}
    storages = (("fp32", M.MPTRAC_FP32), ("bf16", M.MPTRAC_BF16), ("fp16", M.MPTRAC_FP16))
    for name, storage in storages:
        ctx = M.Context(grid, storage, nvars=4)
        ctx.set_launch(2, False)
        work = init.clone()
        sim = Simulation(ctx, at, DT_MET, work, DT, prm, SEED_RNG, SORT_EVERY)

        def one_pass():
            with torch.cuda.stream(stream):
                work.copy_(init)
                sim.run(0.0, PREC_T_END, stream=stream)
        for _ in range(args.warmup):
            one_pass()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            one_pass()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        results[name] = {"ms_per_pass": ms, "particle_steps_per_s": psteps / (ms / 1000.0),
                         "slot_bytes": int(grid.npoints * (16 if storage == M.MPTRAC_FP32 else 8))}
        ctx.close()
        del work, sim
        torch.cuda.empty_cache()
        for diffuse in (True, False):
            subset[(name, diffuse)] = _precision_subset_gpu(M, grid, snaps, storage, sub, diffuse)
    host = [{k: v.cpu().numpy() for k, v in s.items() if k in ("u", "v", "w", "T")} for s in snaps]
    del snaps
    torch.cuda.empty_cache()
    # cpu_baseline leg: the float64 oracle on the subset, from the float32 fields, with and
    # without diffusion; its states are the reference of every error below (the stored-value
    # error of bf16/fp16 plus the float32 arithmetic of every storage)
    t0 = time.perf_counter()
    ref = {d: _precision_oracle(grid, host, sub, d) for d in (True, False)}
    oracle_s = time.perf_counter() - t0
    from oracle import meteo
    for name, _ in storages:
        horizons = {}
        for diffuse in (True, False):
            states, sampled = subset[(name, diffuse)]
            for h in PREC_HORIZONS:
                horizons[f"{'diffusion' if diffuse else 'advection'}_{h / 3600:g}h"] = error_summary(
                    states[h], ref[diffuse][h])
            if diffuse:
                results[name].update(horizons[f"diffusion_{PREC_T_END / 3600:g}h"])
                # sampled met at this run's own final positions vs the float64 sampling of the
                # float32 fields there: the storage's and the interpolation's error alone
                fin = states[PREC_HORIZONS[-1]]
                ms_ = meteo.sample(grid, host[1], DT_MET, host[2], 2 * DT_MET, PREC_T_END, fin["lon"], fin["lat"],
                                   fin["p"])
                for q, var in enumerate(("u", "v", "w", "T")):
                    err = np.abs(sampled[q] - ms_[var])
                    results[name][f"sampled_{var}_abs_median"] = float(np.median(err))
                    results[name][f"sampled_{var}_abs_p99"] = float(np.quantile(err, 0.99))
        results[name]["horizons"] = horizons
        results[name]["speedup_vs_fp32"] = results["fp32"]["ms_per_pass"] / results[name]["ms_per_pass"]
    oracle_psteps = 2 * sub_ids.size * int(round(PREC_T_END / DT))
    line = {"metric": METRIC, "value": results["bf16"]["particle_steps_per_s"], "unit": "particle-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": results["bf16"]["ms_per_pass"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 storage / f32 arithmetic", "data": "synthetic",
            "config": {"workload": "0.3deg 1200x601x137 multiscale Fourier wind (256 modes), u/v/omega/T, "
                                   f"{n} particles, 12 h (240 fused steps), sort every 20; error vs the float64 "
                                   f"oracle on {sub_ids.size} particles, with and without diffusion, at "
                                   "1 h, 6 h and 12 h"},
            "cpu_baseline": {"value": oracle_psteps / oracle_s, "unit": "particle-steps/s", "cores": 1,
                             "kind": "oracle", "sample": f"{sub_ids.size} particles x 12 h, with and without "
                                                         f"diffusion: {oracle_s:.1f} s"},
            "precision": results}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# learned surrogate: train on plain trajectories, then 48 h runs
# --------------------------------------------------------------------------
SURR_SEED, SURR_T_END = 5, 48 * 3600.0


def surrogate_figures(dev, grid, snaps, n, n_train, epochs):
    """Trains the surrogate on ``n_train`` plain 30-minute trajectories, then runs ``n`` particles
    for 48 h three ways: plain midpoint at 180 s (the reference trajectory), plain midpoint at
    1800 s, and the surrogate with the plain fallback; times and great-circle errors."""
    import torch

    import paper_2211_12616_gb300 as M
    from paper_2211_12616_gb300 import learn
    from paper_2211_12616_gb300.simulation import periodic_snapshots
    from workloads import initial_weights, uniform_particles

    at = periodic_snapshots(snaps, DT_MET)
    ctx = M.Context(grid, M.MPTRAC_FP32)
    ctx.set_launch(2, False)
    src = lambda count, seed: uniform_particles(count, grid.plev, SURR_SEED * 100000 + seed, lat_max=80.0)
    t0 = time.perf_counter()
    X, Y = learn.make_dataset(ctx, at, DT_MET, n_train, src)
    t_data = time.perf_counter() - t0
    sur = M.Surrogate(65536)
    sur.set_params(initial_weights(SURR_SEED))
    t0 = time.perf_counter()
    hist, val = learn.train(sur, X, Y, epochs=epochs, batch=8192, lr=2e-3, lr_min=2e-5)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, Y
    torch.cuda.empty_cache()
    st0 = uniform_particles(n, grid.plev, SURR_SEED)
    init = M.Particles.from_numpy(st0, device=dev, meso=False, release=False)
    stream = torch.cuda.Stream(device=dev)
    ws = torch.empty(ctx.sort_workspace_bytes(n), dtype=torch.uint8, device=dev)

    def timed(fn, parts):
        parts.copy_(init)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            out = fn(parts)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    plain, coarse, sur_p = init.clone(), init.clone(), init.clone()
    run_sur = lambda P: learn.run_surrogate(ctx, sur, P, at, DT_MET, 0.0, SURR_T_END, stream=stream, workspace=ws)
    timed(run_sur, sur_p)                                   # first use: set-up outside the timing
    ms_plain, _ = timed(lambda P: learn.run_plain(ctx, P, at, DT_MET, 0.0, SURR_T_END, stream=stream,
                                                  workspace=ws), plain)
    ms_coarse, _ = timed(lambda P: learn.run_plain(ctx, P, at, DT_MET, 0.0, SURR_T_END, dt=learn.DT_SEG,
                                                   stream=stream, workspace=ws), coarse)
    ms_sur, fb = timed(run_sur, sur_p)

    def by_id(parts):
        d = parts.to_numpy()
        o = np.argsort(d["id"])
        return {k: v[o] for k, v in d.items()}

    # the inference kernel alone: one segment over all particles, after the 48 h runs (sorted state)
    fbuf = torch.zeros(n, dtype=torch.uint8, device=dev)
    ctx.load_met(0, 0.0, *at(0.0))
    ctx.load_met(1, DT_MET, *at(DT_MET))
    probe = init.clone()
    ctx.sort(probe, ws)
    inf_ms = []
    for _ in range(4):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sur.advance(ctx, probe, 3600.0, learn.DT_SEG, fbuf, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        inf_ms.append(a.elapsed_time(b))
        probe.copy_(init)
        ctx.sort(probe, ws)
    sur.status()
    t_inf = min(inf_ms[1:]) / 1000.0 / n                       # seconds per particle and segment
    flop = 2 * (176 * 128 + 128 * 128 + 128 * 16)             # the three layers as computed (N of layer 3 padded to 16)
    gather_b = 27 * 2 * 16                                      # 27 nodes x 2 snapshots x 16-byte records
    peak_tf = _bf16_peak()
    l2 = measure_l2_gbs(dev)
    inference = {"ns_per_particle": t_inf * 1e9, "flop_per_particle": flop, "gather_bytes_per_particle": gather_b,
                 "tensor_bound_ns": flop / (peak_tf * 1e12) * 1e9, "gather_bound_ns": gather_b / (l2 * 1e9) * 1e9,
                 "frac_of_gather_bound": gather_b / (l2 * 1e9) / t_inf, "frac_of_tensor_bound": flop / (peak_tf * 1e12) / t_inf,
                 "peaks": f"bf16 {peak_tf:.0f} TFLOP/s (MEASURED_PEAKS.json burst), L2 copy {l2:.0f} GB/s (measured here)"}
    ref = by_id(plain)
    substeps = n * int(round(SURR_T_END / DT))
    runs = {}
    for name, parts, ms in (("plain_dt180", plain, ms_plain), ("midpoint_dt1800", coarse, ms_coarse),
                            ("surrogate", sur_p, ms_sur)):
        got = by_id(parts)
        km = great_circle_km(got["lon"], got["lat"], ref["lon"], ref["lat"])
        dp = np.abs(got["p"] - ref["p"]) / ref["p"]
        runs[name] = {"ms_per_48h": ms, "substep_equivalents_per_s": substeps / (ms / 1000.0),
                      "speedup_vs_plain": ms_plain / ms, "km_median": float(np.median(km)),
                      "km_p99": float(np.quantile(km, 0.99)), "dp_rel_median": float(np.median(dp)),
                      "dp_rel_p99": float(np.quantile(dp, 0.99))}
    runs["surrogate"]["fallback_fraction"] = fb[0].item() / fb[1]
    ctx.close()
    return {"runs": runs, "inference": inference, "train_seconds": t_train, "dataset_seconds": t_data, "epochs": epochs,
            "train_samples": n_train, "particles": n, "train_loss": hist, "val_loss": val,
            "workload": f"surrogate trained on {n_train} plain 30-min trajectories of the 1deg field, "
                        f"{n} particles, 48 h; errors against plain midpoint at 180 s"}


def run_surrogate_bench(args, rank, world):
    import torch

    from workloads import fourier_modes, fourier_snapshot, grid_1deg_60lev

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    grid = grid_1deg_60lev()
    modes = fourier_modes(SEED_FIELD)
    snaps = [fourier_snapshot(grid, modes, h * DT_MET, device=dev, as_numpy=False) for h in range(4)]
    f = surrogate_figures(dev, grid, snaps, args.particles, args.train_samples, args.epochs)
    runs = f["runs"]
    line = {"metric": METRIC, "value": runs["surrogate"]["substep_equivalents_per_s"], "unit": "particle-steps/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": runs["surrogate"]["ms_per_48h"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 MLP / f32",
            "data": "synthetic",
            "config": {"workload": f["workload"] + "; value in 180-s substep equivalents per second",
                       "train_seconds": f["train_seconds"], "dataset_seconds": f["dataset_seconds"],
                       "epochs": f["epochs"], "train_loss": f["train_loss"], "val_loss": f["val_loss"]},
            "surrogate": runs, "inference": f["inference"]}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# next rows: met sampling, particle counts per cell, sedimentation
# --------------------------------------------------------------------------
def run_next(args, rank, world):
    import torch

    import paper_2211_12616_gb300 as M
    from workloads import fourier_modes, fourier_snapshot, grid_1deg_60lev, uniform_particles

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    grid = grid_1deg_60lev()
    modes = fourier_modes(SEED_FIELD, with_T=True)
    f0 = fourier_snapshot(grid, modes, 0.0, device=dev, as_numpy=False)
    f1 = fourier_snapshot(grid, modes, DT_MET, device=dev, as_numpy=False)
    ctx = M.Context(grid, M.MPTRAC_FP32, nvars=4)
    ctx.load_met(0, 0.0, f0["u"], f0["v"], f0["w"], f0["T"])
    ctx.load_met(1, DT_MET, f1["u"], f1["v"], f1["w"], f1["T"])
    n = args.particles if args.particles != N_PART else 10_000_000
    st = uniform_particles(n, grid.plev, 8)
    parts = M.Particles.from_numpy(st, device=dev, meso=False)
    ctx.sort(parts)
    rng = np.random.default_rng(8)
    radius = torch.from_numpy(np.exp(rng.uniform(np.log(1e-7), np.log(2e-5), n)).astype(np.float32)).to(dev)
    density = torch.full((n,), 1500.0, dtype=torch.float32, device=dev)
    p_save = parts.p.clone()

    def timeit(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms_sample = timeit(lambda: ctx.sample_met(parts, 3600.0))
    ms_count = timeit(lambda: ctx.grid_counts(parts))
    ms_sedi = timeit(lambda: (parts.p.copy_(p_save), ctx.sediment(parts, radius, density, 0.0, 180.0, 20)))
    # rooflines from algorithmic bytes: HBM = particle arrays read and written + every slot record
    # of both snapshots read once (an upper bound); L2 = the per-particle corner gather with no reuse
    hbm_peak, hbm_kind = _peaks()
    l2_gbs = measure_l2_gbs(dev)
    cells = grid.nx * grid.ny * grid.nz
    met_b = 2 * cells * 16

    def roof(ms, hbm_b, l2_b=None):
        r = {"hbm_bytes": hbm_b, "hbm_gbs": hbm_b / (ms / 1e3) / 1e9,
             "hbm_frac": hbm_b / (ms / 1e3) / 1e9 / hbm_peak, "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": hbm_kind}
        if l2_b is not None:
            r.update({"l2_bytes": l2_b, "l2_gbs": l2_b / (ms / 1e3) / 1e9, "l2_frac": l2_b / (ms / 1e3) / 1e9 / l2_gbs,
                      "l2_peak_gbs": l2_gbs, "l2_peak_kind": "measured here (copy probe resident in L2)"})
        return r

    line = {"workload": f"next rows on the 1deg x 60-level grid (u, v, omega, T), {n} sorted particles",
            "sample_met": {"ms": ms_sample, "particles_per_s": n / (ms_sample / 1e3),
                           "bytes_per_particle": "HBM 24 (lon, lat, p) + 16 (u, v, omega, T out); "
                                                 "L2 2 snapshots x 8 corners x 16 B",
                           "roofline": roof(ms_sample, 40 * n + met_b, 2 * 8 * 16 * n)},
            "grid_counts": {"ms": ms_count, "particles_per_s": n / (ms_count / 1e3),
                            "bytes_per_particle": "HBM 24 (lon, lat, p) + 4 per cell (zeroed counts)",
                            "cells": grid.npoints, "roofline": roof(ms_count, 24 * n + 4 * cells)},
            "sediment_20_steps": {"ms": ms_sedi, "particle_steps_per_s": 20 * n / (ms_sedi / 1e3),
                                  "bytes_per_particle": "HBM 16 (lon, lat) + 16 (p read, written) + 8 (radius, "
                                                        "density) per launch",
                                  "roofline": roof(ms_sedi, 40 * n + met_b),
                                  "note": "the T corners stay in registers while a particle stays in its cell, so "
                                          "there is no per-step gather; the launch is bound by its arithmetic "
                                          "(T interpolation, viscosity, slip correction per step)"}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--particles", type=int, default=N_PART)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the 16-bit storage, batched and surrogate figures of the default line")
    ap.add_argument("--workload", default="transport", choices=["transport", "batch", "precision", "surrogate", "next"])
    ap.add_argument("--train-samples", type=int, default=10_000_000)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--count-scale", type=float, default=1.0)
    ap.add_argument("--variant", type=int, default=-1,
                    help="fixed launch variant of the fused step (-1: autotuned)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="met storage of the transport workload (fp32: the headline; bf16/fp16 for profiling, "
                         "also reported under forms.storage of the default line)")
    ap.add_argument("--per-thread", type=int, default=1, choices=[1, 2, 4],
                    help="particles per thread of the fused step with a fixed --variant")
    ap.add_argument("--groups", type=int, default=0,
                    help="particle groups on streams of their own (0: the autotuner picks 1, 2 or 3; "
                         "2 with a fixed --variant)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        import __graft_entry__
        __graft_entry__.build()
        if args.workload == "batch":
            run_batch(args, rank, world)
        elif args.workload == "precision":
            run_precision(args, rank, world)
        elif args.workload == "next":
            run_next(args, rank, world)
        elif args.workload == "surrogate":
            if args.particles == N_PART:
                args.particles = 10_000_000
            run_surrogate_bench(args, rank, world)
        else:
            run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
