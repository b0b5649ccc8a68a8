"""The time loop of one transport run through the C ABI.

Mirrors the structure of MPTRAC's main loop (arxiv 2211.12616, Sections 3 and
4.3): whenever the model time leaves the interval spanned by the two loaded
met snapshots the next snapshot is loaded (``read_met`` + update device); the
particles then advance in blocks of ``sort_every`` fused steps (advection,
turbulent and mesoscale diffusion, position rules), and are sorted by met cell
before every block so that each block starts with cell-ordered particles.  The
sort before the first block is a plain ``mptrac_sort``; every later one is
fused into the block before it (``mptrac_step_handoff`` +
``mptrac_sort_handoff``): the block's last launch hands its results to the
sort.

With ``groups`` = G > 1 the particles are split into G contiguous groups, each
sorted and stepped on a stream of its own: a group's sort and the last,
partly filled wave of its step kernel then overlap with the other groups'
steps.  A particle's trajectory does not depend on the other particles or on
their order (counter-based random numbers keyed by particle id), so the
results are those of G = 1 up to the order of the particles in memory.
The met snapshots live in a ring of the context's three slots (snapshot k of
the run in slot k mod 3): the snapshot an interval two ahead needs is loaded
on a stream of its own as soon as every group has finished the interval that
last read the slot it replaces, so loads overlap with the steps.  The groups'
first sorts need no met and overlap the loads of the first two snapshots.

Snapshots that ``snapshot_at`` returns in host memory (pinned, for the copies
to overlap) are prefetched: right after an interval's loads, the snapshot the
next interval needs is copied into one of two device buffers on a copy stream
while the interval computes, and its load then reads the device copy.  The
first two snapshots go the same way, so that the first one's repack overlaps
the second one's copy.

This module only sequences ABI calls.
"""
from __future__ import annotations

import math

import torch

from ._native import Context, DiffParams, Particles


class Simulation:
    def __init__(self, ctx: Context, snapshot_at, dt_met: float, particles: Particles, dt: float,
                 prm: DiffParams, seed: int, sort_every: int = 20, sort: bool = True, groups: int = 1):
        """``snapshot_at(t)`` returns (u, v, w) device tensors of the snapshot at time t."""
        self.ctx, self.snapshot_at, self.dt_met = ctx, snapshot_at, float(dt_met)
        self.parts, self.dt, self.prm, self.seed = particles, float(dt), prm, int(seed)
        self.sort_every, self.do_sort = int(sort_every), bool(sort)
        n, g = particles.n, max(1, min(int(groups), max(particles.n, 1)))
        bounds = [round(q * n / g) for q in range(g + 1)]
        self.groups = [particles.view(bounds[q], bounds[q + 1]) for q in range(g)] if g > 1 else [particles]
        dev = particles.lon.device
        self.workspaces = [torch.empty(ctx.sort_workspace_bytes(v.n), dtype=torch.uint8, device=dev)
                           for v in self.groups] if sort else [None] * g
        self.workspace = self.workspaces[0]
        self._streams = None
        self._load_stream = None
        self._pf = None           # host-snapshot prefetch state (copy stream, device buffers, events)
        self.step_hook = None     # called around every mptrac_step: hook(stage, stream)

    def _on_device(self, fields):
        return all(x is None or (isinstance(x, torch.Tensor) and x.is_cuda) for x in fields)

    def _prefetch(self, t):
        """Copies the host snapshot at time t into the next device buffer on the copy stream."""
        f = self.snapshot_at(t)
        if self._on_device(f) or not all(x is None or isinstance(x, torch.Tensor) for x in f):
            return
        dev = self.parts.lon.device
        if self._pf is None:
            self._pf = {"stream": torch.cuda.Stream(device=dev), "bufs": [None, None], "used": [None, None],
                        "ready": {}, "next": 0}
        pf = self._pf
        b = pf["next"]
        pf["next"] = 1 - b
        if pf["bufs"][b] is None:
            pf["bufs"][b] = [None if x is None else torch.empty(x.shape, dtype=x.dtype, device=dev) for x in f]
        cs = pf["stream"]
        if pf["used"][b] is not None:
            cs.wait_event(pf["used"][b])      # the load that read this buffer has run
        with torch.cuda.stream(cs):
            for dst, src in zip(pf["bufs"][b], f):
                if dst is not None:
                    dst.copy_(src, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(cs)
        pf["ready"][t] = (b, ev)

    def _load(self, ctx, slot, t, stream):
        """Loads the snapshot at time t into ``slot`` on ``stream`` (from its prefetched device copy
        if there is one).  Host snapshots without a prefetch go through the context's staging
        buffer, so the caller keeps such loads on one stream at a time."""
        pf = self._pf
        if pf is not None and t in pf["ready"]:
            b, ev = pf["ready"].pop(t)
            stream.wait_event(ev)
            ctx.load_met(slot, t, *pf["bufs"][b], stream=stream)
            used = torch.cuda.Event()
            used.record(stream)
            pf["used"][b] = used
        else:
            ctx.load_met(slot, t, *self.snapshot_at(t), stream=stream)

    def _group_streams(self, main):
        """(step streams, sort streams): one of each per group; with one group both are ``main``.
        The sorts run at high priority, so that a group's short, latency-bound sort kernels
        take SM slots as the other groups' step blocks retire."""
        if len(self.groups) == 1:
            return [main], [main]
        if self._streams is None:
            dev = self.parts.lon.device
            lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
            self._streams = ([torch.cuda.Stream(device=dev) for _ in self.groups],
                             [torch.cuda.Stream(device=dev, priority=hi) for _ in self.groups])
        return self._streams

    def run(self, t_start: float, t_end: float, stream=None) -> int:
        """Advances from t_start to t_end; returns the number of steps taken.

        t_start and t_end must be multiples of dt_met and the met interval a
        multiple of dt.
        """
        steps_per_iv = int(round(self.dt_met / self.dt))
        if abs(steps_per_iv * self.dt - self.dt_met) > 1e-9 * self.dt_met:
            raise ValueError("the met interval must be a whole number of steps")
        n_iv = int(round((t_end - t_start) / self.dt_met))
        ctx = self.ctx
        dev = self.parts.lon.device
        main = stream if stream is not None else torch.cuda.current_stream(dev)
        gstreams, sstreams = self._group_streams(main)
        if self._load_stream is None:
            self._load_stream = torch.cuda.Stream(device=dev)
        ls = self._load_stream
        T = lambda k: t_start + k * self.dt_met          # snapshot k of the run, in slot k % 3
        loaded = {}                                      # snapshot k -> event after its load
        if n_iv == 0:
            return 0
        # the particles are ready here: the first sorts need no met and overlap the loads
        parts_ready = torch.cuda.Event()
        parts_ready.record(main)
        # snapshots 0 and 1 in stream order; snapshot 2 (a free slot) on the load stream.  Host
        # snapshots 0 and 1 are first both copied on the copy stream, so that the repack of the
        # first overlaps the copy of the second (and the caller's own uploads)
        for k in (0, 1):
            self._prefetch(T(k))
        for k in (0, 1):
            self._load(ctx, k % 3, T(k), main)
        ls.wait_stream(main)
        if n_iv >= 2:
            self._load(ctx, 2, T(2), ls)
            loaded[2] = torch.cuda.Event()
            loaded[2].record(ls)
        for gs in gstreams:
            if gs is not main:
                gs.wait_stream(main)
        step = 0
        sorted_ = False           # particles already sorted by the previous block
        for iv in range(n_iv):
            ta = T(iv)
            if iv + 1 in loaded:  # the interval's later snapshot came from the load stream
                for gs in gstreams:
                    gs.wait_event(loaded[iv + 1])
            if iv + 3 <= n_iv:
                self._prefetch(T(iv + 3))        # host snapshots: copied during this interval
            done = 0
            while done < steps_per_iv:
                cnt = min(self.sort_every, steps_per_iv - done)
                t = ta + done * self.dt
                last = iv == n_iv - 1 and done + cnt >= steps_per_iv   # no block follows
                for parts, ws, gs, ss in zip(self.groups, self.workspaces, gstreams, sstreams):
                    if self.do_sort and not sorted_:
                        if ss is not gs:
                            ss.wait_event(parts_ready)   # the run's first sort: no met needed
                        ctx.sort(parts, ws, stream=ss)
                        if ss is not gs:
                            gs.wait_stream(ss)
                    if self.step_hook:
                        self.step_hook("begin", gs)
                    handoff = self.do_sort and not last
                    if handoff:
                        ctx.step_handoff(parts, t, self.dt, self.prm, self.seed, step, cnt, ws, stream=gs)
                    else:
                        ctx.step(parts, t, self.dt, self.prm, self.seed, step, cnt, stream=gs)
                    if self.step_hook:
                        self.step_hook("end", gs)
                    if handoff:
                        if ss is not gs:
                            ss.wait_stream(gs)
                        ctx.sort_handoff(parts, ws, stream=ss)
                        if ss is not gs:
                            gs.wait_stream(ss)
                sorted_ = self.do_sort
                done += cnt
                step += cnt
            if iv + 3 <= n_iv:
                # snapshot iv + 3 replaces snapshot iv, whose last reader was this interval
                for gs in gstreams:
                    ls.wait_stream(gs)
                self._load(ctx, (iv + 3) % 3, T(iv + 3), ls)
                loaded[iv + 3] = torch.cuda.Event()
                loaded[iv + 3].record(ls)
        for gs in gstreams:
            if gs is not main:
                main.wait_stream(gs)
        main.wait_stream(ls)
        return step


def periodic_snapshots(fields_by_index, dt_met: float):
    """snapshot_at(t) for a list of snapshots repeating with period len(list) * dt_met."""
    n = len(fields_by_index)

    def at(t):
        q = int(math.floor(t / dt_met + 0.5)) % n
        f = fields_by_index[q]
        return f["u"], f["v"], f["w"]
    return at
