"""4D linear interpolation of met fields -- TEST INFRASTRUCTURE ONLY.

``module_advection`` computes trajectories "using given velocities" (Section 3.2);
the velocities come from two met snapshots ``met0``/``met1`` that bracket the
model time (Section 4.1).  The paper gives no interpolation formula; the method
here interpolates linearly in all four dimensions:

* longitude: periodic; x = ((lon - lon0) mod 360) / dlon, i = floor(x) mod nx,
  i+1 wraps to 0, fx = x - floor(x);
* latitude: y = (lat - lat0) / dlat, j = floor(y) clamped to [0, ny-2],
  fy = y - j clamped to [0, 1];
* pressure: p clamped to [min plev, max plev]; with plev strictly decreasing,
  k is the largest index in [0, nz-2] with plev[k] >= p and
  fz = (plev[k] - p) / (plev[k] - plev[k+1]) -- linear in p, not in ln p;
* trilinear in (lon, lat, p) on each snapshot, then linear in time with
  w = (t - t0) / (t1 - t0) in float64.

Fields are float64 arrays [nz][ny][nx].
"""
from __future__ import annotations

import numpy as np


def locate(grid, lon, lat, p):
    """Cell indices and fractions: (i, i1, j, k, fx, fy, fz)."""
    lon = np.asarray(lon, dtype=np.float64)
    lat = np.asarray(lat, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    x = np.mod(lon - grid.lon0, 360.0) / grid.dlon
    fl = np.floor(x)
    fx = x - fl
    i = np.mod(fl.astype(np.int64), grid.nx)
    i1 = np.mod(i + 1, grid.nx)

    y = (lat - grid.lat0) / grid.dlat
    j = np.clip(np.floor(y).astype(np.int64), 0, grid.ny - 2)
    fy = np.clip(y - j, 0.0, 1.0)

    plev = np.asarray(grid.plev, dtype=np.float64)
    pc = np.clip(p, plev[-1], plev[0])
    # number of levels with plev >= pc, minus one  (plev decreasing)
    k = np.searchsorted(-plev, -pc, side="right") - 1
    k = np.clip(k, 0, grid.nz - 2)
    fz = (plev[k] - pc) / (plev[k] - plev[k + 1])
    fz = np.clip(fz, 0.0, 1.0)
    return i, i1, j, k, fx, fy, fz


def corners(f, loc):
    """The 8 corner values of each particle's cell, shape (8, n), order (dk, dj, di)."""
    i, i1, j, k, _, _, _ = loc
    out = []
    for dk in (0, 1):
        for dj in (0, 1):
            for ii in (i, i1):
                out.append(f[k + dk, j + dj, ii])
    return np.stack(out)


def trilinear(f, loc):
    """Trilinear interpolation of field f at located points."""
    _, _, _, _, fx, fy, fz = loc
    c = corners(f, loc)
    # lerp along lon for the four (dk, dj) edges, then along lat, then along p
    e00 = c[0] * (1 - fx) + c[1] * fx      # k,   j
    e01 = c[2] * (1 - fx) + c[3] * fx      # k,   j+1
    e10 = c[4] * (1 - fx) + c[5] * fx      # k+1, j
    e11 = c[6] * (1 - fx) + c[7] * fx      # k+1, j+1
    s0 = e00 * (1 - fy) + e01 * fy
    s1 = e10 * (1 - fy) + e11 * fy
    return s0 * (1 - fz) + s1 * fz


def corner_weights(loc):
    """Trilinear weights of the 8 corners, shape (8, n), same order as ``corners``."""
    _, _, _, _, fx, fy, fz = loc
    out = []
    for wk in (1 - fz, fz):
        for wj in (1 - fy, fy):
            for wi in (1 - fx, fx):
                out.append(wk * wj * wi)
    return np.stack(out)


def corner_variance(f, loc):
    """Subgrid variance: corner values' spread about the interpolated value,
    weighted by the interpolation weights,  sum_c w_c (f_c - sum_c' w_c' f_c')^2.

    At a cell face the weights of the far corners vanish, so the variance is
    continuous across faces (both neighbouring cells give the same value).
    """
    c = corners(f, loc)
    w = corner_weights(loc)
    m = (w * c).sum(axis=0)
    return (w * (c - m) ** 2).sum(axis=0)


def time_weight(t, t0, t1):
    return (np.float64(t) - t0) / (t1 - t0)
