"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package only *generates inputs*: grid descriptions, gridded wind snapshots,
particle releases and the surrogate network's initial weights.  It holds none of the transport method's arithmetic
(no interpolation, no integration, no random-number transform, no sorting), so
both sides of a parity test can draw from it without sharing any step of the
method.  The met data of the paper (netCDF reanalysis read by ``read_met``,
Section 3.1) is not available; the fields here stand in for it with the shapes
and value ranges of the paper's workloads.
"""
from .fields import (Grid, grid_global, grid_2deg_20lev, grid_1deg_60lev, grid_03deg_137lev,
                     cfg1_analytic_wind, cfg1_snapshot, fourier_modes, fourier_snapshot)
from .particles import uniform_particles, column_releases, Releases
from .network import initial_weights

__all__ = [
    "Grid", "grid_global", "grid_2deg_20lev", "grid_1deg_60lev", "grid_03deg_137lev",
    "cfg1_analytic_wind", "cfg1_snapshot", "fourier_modes", "fourier_snapshot",
    "uniform_particles", "column_releases", "Releases", "initial_weights",
]
