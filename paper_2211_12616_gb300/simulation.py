"""The time loop of one transport run through the C ABI.

Mirrors the structure of MPTRAC's main loop (arxiv 2211.12616, Sections 3 and
4.3): whenever the model time leaves the interval spanned by the two loaded
met snapshots the next snapshot is loaded (``read_met`` + update device); the
particles then advance in blocks of ``sort_every`` fused steps (advection,
turbulent and mesoscale diffusion, position rules), and are sorted by met cell
before every block so that each block starts with cell-ordered particles.

All work is enqueued on one CUDA stream; this module only sequences ABI calls.
"""
from __future__ import annotations

import math

import torch

from ._native import Context, DiffParams, Particles


class Simulation:
    def __init__(self, ctx: Context, snapshot_at, dt_met: float, particles: Particles, dt: float,
                 prm: DiffParams, seed: int, sort_every: int = 20, sort: bool = True):
        """``snapshot_at(t)`` returns (u, v, w) device tensors of the snapshot at time t."""
        self.ctx, self.snapshot_at, self.dt_met = ctx, snapshot_at, float(dt_met)
        self.parts, self.dt, self.prm, self.seed = particles, float(dt), prm, int(seed)
        self.sort_every, self.do_sort = int(sort_every), bool(sort)
        self.workspace = torch.empty(ctx.sort_workspace_bytes(particles.n), dtype=torch.uint8,
                                     device=particles.lon.device) if sort else None
        self.step_hook = None     # called around every mptrac_step: hook(stage, stream)

    def run(self, t_start: float, t_end: float, stream=None) -> int:
        """Advances from t_start to t_end; returns the number of steps taken.

        t_start and t_end must be multiples of dt_met and the met interval a
        multiple of dt.
        """
        steps_per_iv = int(round(self.dt_met / self.dt))
        if abs(steps_per_iv * self.dt - self.dt_met) > 1e-9 * self.dt_met:
            raise ValueError("the met interval must be a whole number of steps")
        n_iv = int(round((t_end - t_start) / self.dt_met))
        ctx, slots = self.ctx, {}
        step = 0
        for iv in range(n_iv):
            ta = t_start + iv * self.dt_met
            tb = ta + self.dt_met
            for t, keep in ((ta, tb), (tb, ta)):
                if t in slots.values():
                    continue
                free = [q for q in (0, 1) if q not in slots]
                slot = free[0] if free else (0 if slots[0] != keep else 1)
                ctx.load_met(slot, t, *self.snapshot_at(t), stream=stream)
                slots[slot] = t
            done = 0
            while done < steps_per_iv:
                cnt = min(self.sort_every, steps_per_iv - done)
                if self.do_sort:
                    ctx.sort(self.parts, self.workspace, stream=stream)
                t = ta + done * self.dt
                if self.step_hook:
                    self.step_hook("begin", stream)
                ctx.step(self.parts, t, self.dt, self.prm, self.seed, step, cnt, stream=stream)
                if self.step_hook:
                    self.step_hook("end", stream)
                done += cnt
                step += cnt
        return step


def periodic_snapshots(fields_by_index, dt_met: float):
    """snapshot_at(t) for a list of snapshots repeating with period len(list) * dt_met."""
    n = len(fields_by_index)

    def at(t):
        q = int(math.floor(t / dt_met + 0.5)) % n
        f = fields_by_index[q]
        return f["u"], f["v"], f["w"]
    return at
