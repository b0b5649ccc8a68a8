"""Batched runs: many releases in one particle array, one CUDA graph per met interval.

MPTRAC's time loop advances every air parcel of a run together, with
``module_timesteps`` giving each parcel a zero step outside its release window
(arxiv 2211.12616, Section 4.3).  Here all releases of a batch share one
structure-of-arrays; the release table drives the per-step activity mask in the
fused step kernel, and the release-aware sort (``mptrac_sort_at``) moves the
parcels of finished releases behind the active ones so that whole warps stay
busy.  The work of one met interval -- loading the next snapshot, then blocks
of ``sort_every`` fused steps each preceded by a sort -- is captured once into a
CUDA graph and replayed, so a 72 h run is a dozen graph launches instead of
hundreds of kernel launches from Python.

The launch configuration (``variant``, ``persistent``, ``per_thread``) and ``sort_every`` change
only the schedule, never the results; ``autotune`` picks them by timing.
"""
from __future__ import annotations

import torch

from ._native import Context, DiffParams, Particles


class BatchedRun:
    def __init__(self, ctx: Context, snapshot_at, dt_met: float, particles: Particles,
                 t_start_rel, t_end_rel, dt: float, prm: DiffParams, seed: int,
                 sort_every: int = 20, variant: int = 0, persistent: bool = True, per_thread: int = 1):
        self.ctx, self.snapshot_at, self.dt_met = ctx, snapshot_at, float(dt_met)
        self.parts, self.dt, self.prm, self.seed = particles, float(dt), prm, int(seed)
        self.sort_every, self.variant, self.persistent = int(sort_every), int(variant), bool(persistent)
        self.per_thread = int(per_thread)
        ctx.set_releases(t_start_rel, t_end_rel)
        self.workspace = torch.empty(ctx.sort_workspace_bytes(particles.n), dtype=torch.uint8,
                                     device=particles.lon.device)
        self.graphs = []
        self.step_hook = None

    def _plan(self, t_start: float, t_end: float):
        """Per interval: the snapshots to load (slot, time) and the step blocks (t, step0, count)."""
        steps_per_iv = int(round(self.dt_met / self.dt))
        if abs(steps_per_iv * self.dt - self.dt_met) > 1e-9 * self.dt_met:
            raise ValueError("the met interval must be a whole number of steps")
        n_iv = int(round((t_end - t_start) / self.dt_met))
        slots, plan, step = {}, [], 0
        for iv in range(n_iv):
            ta = t_start + iv * self.dt_met
            tb = ta + self.dt_met
            loads = []
            for t, keep in ((ta, tb), (tb, ta)):
                if t in slots.values():
                    continue
                free = [q for q in (0, 1) if q not in slots]
                slot = free[0] if free else (0 if slots[0] != keep else 1)
                loads.append((slot, t))
                slots[slot] = t
            blocks, done = [], 0
            while done < steps_per_iv:
                cnt = min(self.sort_every, steps_per_iv - done)
                blocks.append((ta + done * self.dt, step, cnt))
                done += cnt
                step += cnt
            plan.append((loads, blocks))
        return plan

    def _enqueue(self, loads, blocks, stream):
        ctx = self.ctx
        ctx.set_launch(self.variant, self.persistent, self.per_thread)
        for slot, t in loads:
            ctx.load_met(slot, t, *self.snapshot_at(t), stream=stream)
        for t, step0, cnt in blocks:
            ctx.sort_at(self.parts, t, self.workspace, stream=stream)
            if self.step_hook:
                self.step_hook("begin", stream)
            ctx.step(self.parts, t, self.dt, self.prm, self.seed, step0, cnt, stream=stream)
            if self.step_hook:
                self.step_hook("end", stream)

    def run_eager(self, t_start: float, t_end: float, stream=None):
        """Enqueues the whole run directly (no graphs)."""
        for loads, blocks in self._plan(t_start, t_end):
            self._enqueue(loads, blocks, stream)

    def capture(self, t_start: float, t_end: float, stream: torch.cuda.Stream):
        """Captures one CUDA graph per met interval (the work is not executed)."""
        self.graphs = []
        for loads, blocks in self._plan(t_start, t_end):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
                self._enqueue(loads, blocks, stream)
            self.graphs.append(g)
        return self.graphs

    def replay(self):
        for g in self.graphs:
            g.replay()
