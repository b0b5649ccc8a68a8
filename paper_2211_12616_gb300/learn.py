"""Training data, training loop and runs of the learned displacement surrogate.

Everything numeric runs in libmptrac's kernels (features, plain midpoint
trajectories, targets, column statistics, BF16 forward/backward, Adam, the
surrogate segment and the masked fallback); this module sequences the calls
and moves tensors around.

* ``make_dataset``: particles uniform in lon, lat (|lat| <= 80) and ln p start
  at several times inside each met interval; their features are taken at the
  start, then the plain integrator (advection only) runs 10 substeps of 180 s
  and the displacement becomes the target.
* ``train``: standardises features and targets with their column statistics,
  then runs Adam on shuffled mini-batches with a cosine learning-rate decay
  (``mptrac_surr_train_epoch``: one library call per epoch).
* ``run_surrogate`` / ``run_plain``: 30-minute segments by the network (with
  the plain fallback), or by the plain integrator -- 10 substeps of 180 s (the
  reference trajectory), or one midpoint step of 30 minutes (``dt=DT_SEG``, the cheapest plain
  alternative: two wind evaluations per segment).
"""
from __future__ import annotations

import math

import torch

from ._native import (Context, Particles, Surrogate, advect_masked, colstats, surr_features,
                      surr_targets)

DT = 180.0
SEG_STEPS = 10
DT_SEG = DT * SEG_STEPS


def _load_interval(ctx, snapshot_at, ta, tb, stream=None):
    ctx.load_met(0, ta, *snapshot_at(ta), stream=stream)
    ctx.load_met(1, tb, *snapshot_at(tb), stream=stream)


def make_dataset(ctx: Context, snapshot_at, dt_met: float, n_samples: int, particle_source,
                 n_intervals: int = 4, stride_steps: int = 10, stream=None):
    """Device tensors X [n][176], Y [n][3] from plain trajectories.

    ``particle_source(count, seed)`` returns a particle dict (lon, lat, p, id).
    """
    steps_per_iv = int(round(dt_met / DT))
    offsets = list(range(0, steps_per_iv - SEG_STEPS + 1, stride_steps))
    groups = [(iv, off) for iv in range(n_intervals) for off in offsets]
    per = int(math.ceil(n_samples / len(groups)))
    X = torch.empty(per * len(groups), 176, dtype=torch.float32, device="cuda")
    Y = torch.empty(per * len(groups), 3, dtype=torch.float32, device="cuda")
    row = 0
    for gi, (iv, off) in enumerate(groups):
        ta, tb = iv * dt_met, (iv + 1) * dt_met
        if off == offsets[0]:
            _load_interval(ctx, snapshot_at, ta, tb, stream)
        t = ta + off * DT
        st = particle_source(per, 1000 + gi)
        p0 = Particles.from_numpy(st, meso=False, release=False)
        surr_features(ctx, p0, t, out=X[row:row + per], stream=stream)
        p1 = p0.clone()
        ctx.advect(p1, t, DT, SEG_STEPS, stream=stream)
        surr_targets(p0, p1, out=Y[row:row + per], stream=stream)
        row += per
    torch.cuda.synchronize()
    return X[:n_samples], Y[:n_samples]


def train(surr: Surrogate, X: torch.Tensor, Y: torch.Tensor, epochs: int = 4, batch: int = 8192,
          lr: float = 2e-3, lr_min: float = 2e-5, val_frac: float = 0.1, seed: int = 0, log=None):
    """Trains in place; returns (train_loss_per_epoch, val_loss)."""
    n = X.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    perm = torch.randperm(n, generator=g, device="cuda")
    X, Y = X[perm], Y[perm]
    n_val = int(n * val_frac)
    Xt, Yt, Xv, Yv = X[n_val:], Y[n_val:], X[:n_val], Y[:n_val]
    mu_x, sd_x = colstats(Xt)      # constant (padding) columns come back with sd 1
    mu_y, sd_y = colstats(Yt)
    surr.set_norm(mu_x, sd_x, mu_y, sd_y)
    nt = Xt.shape[0]
    steps_per_epoch = nt // batch
    total = steps_per_epoch * epochs
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    history = []
    for ep in range(epochs):
        loss.zero_()
        order = torch.randperm(nt, generator=g, device="cuda")
        Xe, Ye = Xt[order], Yt[order]
        if steps_per_epoch:   # the epoch's Adam steps and their learning rates: one library call
            surr.train_epoch(Xe, Ye, batch, lr, lr_min, ep * steps_per_epoch, total, loss)
        history.append(loss.item() / max(steps_per_epoch, 1))
        if log:
            log(f"epoch {ep}: train loss {history[-1]:.5f}")
    return history, evaluate(surr, Xv, Yv, batch)


def evaluate(surr: Surrogate, X: torch.Tensor, Y: torch.Tensor, batch: int = 8192) -> float:
    """Mean squared error in normalised units."""
    total, n = 0.0, X.shape[0]
    for o in range(0, n, batch):
        c = min(batch, n - o)
        total += surr.grads(X[o:o + c], Y[o:o + c]).item() * c
    return total / max(n, 1)


def run_surrogate(ctx: Context, surr: Surrogate, parts: Particles, snapshot_at, dt_met: float, t_start: float,
                  t_end: float, stream=None, workspace=None):
    """Surrogate segments with the plain fallback; returns (device count of fallback particle-segments,
    particle-segments).

    Particles are sorted by met cell at the start of every met interval, which also groups the
    fallback particles (poles, rare wind patterns) into whole warps of the masked plain kernel.
    """
    fallback = torch.zeros(parts.n, dtype=torch.uint8, device=parts.lon.device)
    if workspace is None:
        workspace = torch.empty(ctx.sort_workspace_bytes(parts.n), dtype=torch.uint8, device=parts.lon.device)
    segs_per_iv = int(round(dt_met / DT_SEG))
    n_iv = int(round((t_end - t_start) / dt_met))
    count = torch.zeros(1, dtype=torch.int64, device=parts.lon.device)   # fallback particle-segments
    for iv in range(n_iv):
        ta = t_start + iv * dt_met
        _load_interval(ctx, snapshot_at, ta, ta + dt_met, stream)
        ctx.sort(parts, workspace, stream=stream)
        for sg in range(segs_per_iv):
            t = ta + sg * DT_SEG
            surr.advance(ctx, parts, t, DT_SEG, fallback, count, stream=stream)
            advect_masked(ctx, parts, fallback, t, DT, SEG_STEPS, stream=stream)
    return count, parts.n * segs_per_iv * n_iv


def run_plain(ctx: Context, parts: Particles, snapshot_at, dt_met: float, t_start: float, t_end: float,
              dt: float = DT, stream=None, workspace=None):
    """Plain midpoint advection over [t_start, t_end] with step dt (the reference trajectory at dt = 180 s);
    particles sorted by met cell at the start of every met interval, like ``run_surrogate``."""
    if workspace is None:
        workspace = torch.empty(ctx.sort_workspace_bytes(parts.n), dtype=torch.uint8, device=parts.lon.device)
    n_iv = int(round((t_end - t_start) / dt_met))
    steps = int(round(dt_met / dt))
    for iv in range(n_iv):
        ta = t_start + iv * dt_met
        _load_interval(ctx, snapshot_at, ta, ta + dt_met, stream)
        ctx.sort(parts, workspace, stream=stream)
        ctx.advect(parts, ta, dt, steps, stream=stream)
