"""Sampling met data along trajectories and gridding particles -- TEST INFRASTRUCTURE ONLY.

* ``sample``: ``module_meteo`` (Section 3.2) samples the met data along the
  trajectories at fixed times; here the four stored variables (u, v, omega, T)
  are interpolated at the particle positions with the 4D linear rule of
  ``interp`` (the one the advection uses).
* ``grid_counts``: ``write_grid`` (Section 3.3) writes gridded data derived from
  the particles; here the number of particles in every met cell, with the cell
  rule of the sort (key = (j nx + i) nz + k).
"""
from __future__ import annotations

import numpy as np

from . import interp
from .sort import cell_keys

VARS = ("u", "v", "w", "T")


def sample(grid, f0, t0, f1, t1, t, lon, lat, p):
    """dict var -> float64 values at the positions, time-interpolated between f0 (t0) and f1 (t1)."""
    loc = interp.locate(grid, lon, lat, p)
    w = interp.time_weight(t, t0, t1)
    out = {}
    for v in VARS:
        if v not in f0:
            continue
        a = interp.trilinear(np.asarray(f0[v], np.float64), loc)
        b = interp.trilinear(np.asarray(f1[v], np.float64), loc)
        out[v] = (1 - w) * a + w * b
    return out


def grid_counts(grid, lon, lat, p):
    """Particles per met cell, an array of nx*ny*nz counts indexed by the cell key."""
    keys = cell_keys(grid, lon, lat, p).astype(np.int64)
    return np.bincount(keys, minlength=grid.nx * grid.ny * grid.nz).astype(np.uint32)
