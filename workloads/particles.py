"""Seeded particle releases (inputs only).

The paper reads initial air-parcel positions with ``read_atm`` (Section 3.1) into
the ``atm_t`` structure of per-parcel arrays (time, p, lon, lat, ...; Section 4.4).
Here particles are drawn from a seed:

* ``uniform_particles`` -- uniform in longitude and latitude (degrees, not area
  weighted) and uniform in ln p over the grid's pressure range.
* ``column_releases`` -- independent vertical line sources (1-20 km altitude,
  p = 1013.25 hPa exp(-z / 7 km)) at random longitude/latitude, with particle
  counts log-uniform in [1e3, 1e6] and release durations uniform in [6, 72] h,
  all starting at t = 0.

Positions are float64 (lon in [0, 360), lat in [-90, 90], p in Pa); ``id`` is a
unique uint32 per particle and ``release`` the uint32 index of its release.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def uniform_particles(n: int, plev: np.ndarray, seed: int, lat_max: float = 90.0,
                      id0: int = 0) -> dict:
    rng = np.random.default_rng(seed)
    lon = rng.uniform(0.0, 360.0, n)
    lat = rng.uniform(-lat_max, lat_max, n)
    lo, hi = np.log(plev.min()), np.log(plev.max())
    p = np.exp(rng.uniform(lo, hi, n))
    p = np.clip(p, plev.min(), plev.max())
    return {
        "lon": lon, "lat": lat, "p": p,
        "id": (np.arange(n, dtype=np.uint64) + id0).astype(np.uint32),
        "release": np.zeros(n, dtype=np.uint32),
    }


@dataclass
class Releases:
    t_start: np.ndarray   # [s], float64 per release
    t_end: np.ndarray     # [s], float64 per release
    counts: np.ndarray    # particles per release
    particles: dict       # lon, lat, p, id, release


def column_releases(n_releases: int, seed: int, count_min: float = 1e3, count_max: float = 1e6,
                    dur_min_h: float = 6.0, dur_max_h: float = 72.0,
                    z_min: float = 1000.0, z_max: float = 20000.0,
                    count_scale: float = 1.0) -> Releases:
    """Vertical line-source releases; ``count_scale`` shrinks every count (tests)."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(np.log(count_min), np.log(count_max), n_releases))
    counts = np.maximum(1, np.round(counts * count_scale)).astype(np.int64)
    dur = rng.uniform(dur_min_h, dur_max_h, n_releases) * 3600.0
    lon_r = rng.uniform(0.0, 360.0, n_releases)
    lat_r = rng.uniform(-90.0, 90.0, n_releases)
    parts = {"lon": [], "lat": [], "p": [], "release": []}
    for r in range(n_releases):
        c = int(counts[r])
        z = rng.uniform(z_min, z_max, c)
        parts["lon"].append(np.full(c, lon_r[r]))
        parts["lat"].append(np.full(c, lat_r[r]))
        parts["p"].append(101325.0 * np.exp(-z / 7000.0))
        parts["release"].append(np.full(c, r, dtype=np.uint32))
    out = {k: np.concatenate(v) for k, v in parts.items()}
    out["id"] = np.arange(out["lon"].size, dtype=np.uint32)
    return Releases(np.zeros(n_releases), dur, counts, out)
