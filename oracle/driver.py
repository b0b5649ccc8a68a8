"""Multi-interval run of the oracle -- TEST INFRASTRUCTURE ONLY.

The time loop of MPTRAC (Sections 3 and 4.3 of the paper): for each pair of
consecutive met snapshots (t_a, t_b) the particles take (t_b - t_a) / dt steps
of the fused chain (``transport.step``).  Sorting changes only the order of the
particle arrays, never their values, so this float64 run does not sort;
results are compared per particle id.
"""
from __future__ import annotations

from . import met as omet
from . import transport as tr


def run_schedule(grid, snapshot_at, dt_met, state, t_start, t_end, dt, prm, seed,
                 storage=omet.FP32, windows=None, mode="step"):
    """``snapshot_at(t)`` returns a dict of float32 fields u, v, w at time t."""
    st = tr.copy_state(state)
    steps_per_iv = int(round(dt_met / dt))
    n_iv = int(round((t_end - t_start) / dt_met))
    step = 0
    for iv in range(n_iv):
        ta = t_start + iv * dt_met
        tb = ta + dt_met
        met = tr.Met(grid, ta, omet.stored_fields(snapshot_at(ta), storage),
                     tb, omet.stored_fields(snapshot_at(tb), storage))
        if mode == "advect":
            st = tr.advect(met, st, ta, dt, steps_per_iv, windows=windows)
        else:
            st = tr.step(met, st, ta, dt, prm, seed, step, steps_per_iv, windows=windows)
        step += steps_per_iv
    return st
