"""Autotuner for the launch schedule of the transport kernels.

The knobs change only how the work is scheduled, never the result (tested
bit-exact): the launch variant of the fused step kernel (threads per block,
register cap, corner cache in registers or shared memory), the schedule of the
blocks (one wave of persistent blocks, or 1, 2 or 4 particles per thread), and
the number of fused steps between two sorts.  Each candidate is timed with
CUDA events on a representative slice of the real workload (one met interval
from the real initial state) and the fastest is kept; results can be cached in
a JSON file keyed by the device and the workload.
"""
from __future__ import annotations

import itertools
import json
import os

import torch

VARIANTS = (0, 1, 2, 3, 4, 5, 6)   # 64 to 512 threads per block, register or shared-memory corner cache
PERSISTENT = (False, True)
PER_THREAD = (1, 2, 4)
SORT_EVERY = (5, 10, 20, 40, 120)


def candidates(variants=VARIANTS, persistent=PERSISTENT, sort_every=SORT_EVERY, groups=(1,),
               per_thread=PER_THREAD):
    """Schedules to try; ``groups`` is the number of particle groups on streams of their own
    (used by runs that support it).  A persistent launch has no particles-per-thread count
    (``per_thread`` 1)."""
    blocks = [(p, k) for p in persistent for k in (per_thread if not p else (1,))]
    return [{"variant": v, "persistent": p, "per_thread": k, "sort_every": s, "groups": g}
            for v, (p, k), s, g in itertools.product(variants, blocks, sort_every, groups)]


def _time(fn, reset, stream, repeats):
    best = float("inf")
    for _ in range(repeats):
        reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def autotune(make_run, reset, cands, stream, repeats=2, cache_path=None, cache_key=None):
    """Returns (best_config, {config_str: ms}).

    make_run(cfg) -> callable enqueuing the timed work on `stream`;
    reset() restores the initial state (not timed).
    """
    if cache_path and cache_key and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if cache_key in cache:
            return cache[cache_key]["best"], cache[cache_key]["timings"]
    timings = {}
    for cfg in cands:
        run = make_run(cfg)
        reset()
        run()                       # warm-up (first-touch, occupancy queries)
        ms = _time(run, reset, stream, repeats)
        timings[json.dumps(cfg, sort_keys=True)] = ms
    best = json.loads(min(timings, key=timings.get))
    if cache_path and cache_key:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[cache_key] = {"best": best, "timings": timings}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, timings
