"""Particle sorting by met cell -- TEST INFRASTRUCTURE ONLY.

The paper lists the sorting modules among the parts of MPTRAC that still wait
for the multi-GPU port (Section 6).  The method reorders all per-particle
arrays so that particles in the same met cell become neighbours in memory:

* key = (j * nx + i) * nz + k, the (i, j, k) of ``interp.locate`` -- the same
  order as the device's [lat][lon][level] met records;
* a stable sort by key (equal keys keep their previous relative order);
* every per-particle array is permuted the same way.
"""
from __future__ import annotations

import numpy as np

from . import interp


def cell_keys(grid, lon, lat, p) -> np.ndarray:
    i, _, j, k, _, _, _ = interp.locate(grid, lon, lat, p)
    return ((j * grid.nx + i) * grid.nz + k).astype(np.uint32)


def sort_permutation(grid, state) -> np.ndarray:
    keys = cell_keys(grid, state["lon"], state["lat"], state["p"])
    return np.argsort(keys, kind="stable")


def sort_state(grid, state) -> dict:
    perm = sort_permutation(grid, state)
    return {k: np.asarray(v)[perm] for k, v in state.items()}


def sort_permutation_at(grid, state, t, windows):
    """Stable sort by cell key, with particles of releases inactive at time t last.

    A release r is active at t if t_start[r] <= t < t_end[r]; particles whose
    release index is outside the table are inactive.  Inactive particles get a
    key above every cell key, so they follow all active particles in their
    previous relative order.
    """
    keys = cell_keys(grid, state["lon"], state["lat"], state["p"]).astype(np.int64)
    ts, te = (np.asarray(a, dtype=np.float64) for a in windows)
    rel = np.asarray(state["release"]).astype(np.int64)
    inside = rel < ts.size
    r = np.where(inside, rel, 0)
    active = inside & (t >= ts[r]) & (t < te[r])
    keys = np.where(active, keys, grid.nx * grid.ny * grid.nz)
    return np.argsort(keys, kind="stable")
