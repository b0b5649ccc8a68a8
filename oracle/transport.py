"""Trajectory time stepping -- TEST INFRASTRUCTURE ONLY.

Restates, in float64 and one particle-vectorised step at a time, the chain of
modules the paper runs inside its time loop (Sections 3.2 and 4.3):
``module_timesteps`` -> ``module_advection`` -> ``module_diffusion_turb`` ->
``module_diffusion_meso`` -> ``module_position``.  The paper gives no numerics,
so the following readings are used (each is also listed with its reason in the
design notes of the repository):

* Time-step mask: a particle of release r moves at step n only if
  t_start[r] <= t + n dt < t_end[r]; otherwise it is left untouched.
* Advection: explicit midpoint on the sphere (angles in degrees,
  R = 6 371 000 m):  x* = x + dt/2 V(x, t);  x' = x + dt V(x*, t + dt/2), where
  dlon = u dt / (R cos(lat)) * 180/pi, dlat = v dt / R * 180/pi, dp = omega dt.
  The second stage uses cos(lat) of the midpoint x*.  x* is brought back into
  the domain (same rules as ``module_position``) before it is used.
  cos(lat) means max(|cos(lat)|, cos(89.999 deg)).
* Turbulent diffusion: horizontal displacements sqrt(2 Dx dt) xi metres east
  and north, vertical sqrt(2 Dz dt) xi metres converted to pressure as
  dp = -p dz / H with H = 7000 m.
* Mesoscale diffusion: a per-particle AR(1) wind perturbation
  u' <- r u' + sqrt(1 - r^2) f sigma_u xi with r = 1 - 2 dt / (t1 - t0)
  (clamped to [0, 1]) and sigma_u^2 the subgrid variance of u: on each
  snapshot the spread of the 8 cell-corner values about the interpolated
  value, weighted by the interpolation weights (continuous across cell
  faces), then interpolated linearly in time; same for v and omega.
  The displacement is u' dt (converted like advection).  The corners are those
  of the first wind evaluation of the step (at x_n, t_n).
* Diffusion displacements (turbulent + mesoscale) are converted at the
  post-advection position: cos(lat) and p of x after advection.
* Random numbers: ``philox.normals4`` with counter (id, step0 + n, stream,
  release).  The normals of stream 0 and then stream 1 are used in order:
  turbulent takes z0..z2 of stream 0, mesoscale z3 of stream 0 and z0, z1 of
  stream 1 (z2, z3 of stream 1 are not used).
* Position boundaries (``module_position``): lat > 90 -> 180 - lat,
  lat < -90 -> -180 - lat, each with lon + 180; lon wrapped into
  [lon0, lon0 + 360); p clamped to [min plev, max plev].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import interp, philox

R_EARTH = 6371000.0
RAD2DEG = 180.0 / np.pi
COS_FLOOR = np.cos(np.radians(89.999))
H_SCALE = 7000.0


@dataclass
class DiffParams:
    dx: float = 50.0        # horizontal turbulent diffusivity [m^2/s]
    dz: float = 0.1         # vertical turbulent diffusivity [m^2/s]
    meso_f: float = 0.16    # mesoscale scaling factor f
    scale_height: float = H_SCALE
    turb: bool = True
    meso: bool = True


class Met:
    """Two gridded snapshots (float64 fields [nz][ny][nx]) at times t0 < t1."""

    def __init__(self, grid, t0, f0, t1, f1):
        self.grid, self.t0, self.t1 = grid, float(t0), float(t1)
        self.f0 = {k: np.asarray(f0[k], dtype=np.float64) for k in ("u", "v", "w")}
        self.f1 = {k: np.asarray(f1[k], dtype=np.float64) for k in ("u", "v", "w")}
        self.pmin, self.pmax = float(np.min(grid.plev)), float(np.max(grid.plev))
        self.lon0 = float(grid.lon0)

    def wind(self, lon, lat, p, t, sigma=False):
        loc = interp.locate(self.grid, lon, lat, p)
        w = interp.time_weight(t, self.t0, self.t1)
        out = [(1 - w) * interp.trilinear(self.f0[c], loc) + w * interp.trilinear(self.f1[c], loc)
               for c in ("u", "v", "w")]
        if sigma:
            out += [(1 - w) * interp.corner_variance(self.f0[c], loc)
                    + w * interp.corner_variance(self.f1[c], loc) for c in ("u", "v", "w")]
        return out


class AnalyticMet:
    """Wind given by a function ``func(lon, lat, p, t) -> (u, v, omega)``.

    Used for closed-form checks; the subgrid variance is zero.
    """

    def __init__(self, func, t0, t1, pmin, pmax, lon0=0.0):
        self.func, self.t0, self.t1 = func, float(t0), float(t1)
        self.pmin, self.pmax, self.lon0 = float(pmin), float(pmax), float(lon0)

    def wind(self, lon, lat, p, t, sigma=False):
        u, v, w = self.func(lon, lat, np.clip(p, self.pmin, self.pmax), t)
        out = [np.asarray(u, float), np.asarray(v, float), np.asarray(w, float)]
        if sigma:
            out += [np.zeros_like(out[0])] * 3
        return out


def coslat(lat):
    return np.maximum(np.abs(np.cos(np.radians(lat))), COS_FLOOR)


def position_bc(lon, lat, p, lon0, pmin, pmax):
    """``module_position``: reflect over the poles, wrap longitude, clamp pressure."""
    lon = np.array(lon, dtype=np.float64, copy=True)
    lat = np.array(lat, dtype=np.float64, copy=True)
    north = lat > 90.0
    lat[north] = 180.0 - lat[north]
    lon[north] += 180.0
    south = lat < -90.0
    lat[south] = -180.0 - lat[south]
    lon[south] += 180.0
    r = np.mod(lon - lon0, 360.0)
    r = np.where(r >= 360.0, r - 360.0, r)
    lon = lon0 + r
    p = np.clip(p, pmin, pmax)
    return lon, lat, p


def _windows_active(state, t_n, windows):
    if windows is None:
        return np.ones(state["lon"].shape, dtype=bool)
    ts, te = windows
    rel = state["release"].astype(np.int64)
    return (t_n >= ts[rel]) & (t_n < te[rel])


def _midpoint(met, lon, lat, p, t, dt, sigma):
    ev = met.wind(lon, lat, p, t, sigma=sigma)
    u, v, w = ev[:3]
    c = coslat(lat)
    lon_s = lon + 0.5 * dt * u / (R_EARTH * c) * RAD2DEG
    lat_s = lat + 0.5 * dt * v / R_EARTH * RAD2DEG
    p_s = p + 0.5 * dt * w
    lon_s, lat_s, p_s = position_bc(lon_s, lat_s, p_s, met.lon0, met.pmin, met.pmax)
    u2, v2, w2 = met.wind(lon_s, lat_s, p_s, t + 0.5 * dt)
    c2 = coslat(lat_s)
    lon_n = lon + dt * u2 / (R_EARTH * c2) * RAD2DEG
    lat_n = lat + dt * v2 / R_EARTH * RAD2DEG
    p_n = p + dt * w2
    return lon_n, lat_n, p_n, (ev[3:] if sigma else None)


def _diffusion(met, st, sel, lon, lat, p, s2, step, seed, dt, prm):
    """Turbulent + mesoscale displacement of the particles ``sel`` at (lon, lat, p)."""
    pid, rel = st["id"][sel], st["release"][sel]
    dlon = np.zeros_like(lon)
    dlat = np.zeros_like(lon)
    dp = np.zeros_like(lon)
    if prm.turb or prm.meso:
        z0, z1, z2, z3 = philox.normals4(pid, step, philox.STREAM_TURB, rel, seed)
    if prm.turb:
        sh = np.sqrt(2.0 * prm.dx * dt)
        sv = np.sqrt(2.0 * prm.dz * dt)
        dlon += sh * z0
        dlat += sh * z1
        dp += -p * (sv * z2) / prm.scale_height
    if prm.meso:
        m1, m2, _, _ = philox.normals4(pid, step, philox.STREAM_MESO, rel, seed)
        m0 = z3
        r = np.clip(1.0 - 2.0 * dt / (met.t1 - met.t0), 0.0, 1.0)
        a = np.sqrt(1.0 - r * r) * prm.meso_f
        up = r * st["up"][sel] + a * np.sqrt(s2[0]) * m0
        vp = r * st["vp"][sel] + a * np.sqrt(s2[1]) * m1
        wp = r * st["wp"][sel] + a * np.sqrt(s2[2]) * m2
        st["up"][sel], st["vp"][sel], st["wp"][sel] = up, vp, wp
        dlon += up * dt
        dlat += vp * dt
        dp += wp * dt
    c = coslat(lat)
    return (lon + dlon / (R_EARTH * c) * RAD2DEG, lat + dlat / R_EARTH * RAD2DEG, p + dp)


def copy_state(state):
    st = {k: np.array(v, copy=True) for k, v in state.items()}
    for k in ("lon", "lat", "p"):
        st[k] = st[k].astype(np.float64)
    n = st["lon"].shape[0]
    for k in ("up", "vp", "wp"):
        st[k] = np.asarray(st.get(k, np.zeros(n)), dtype=np.float64).copy()
    if "release" not in st:
        st["release"] = np.zeros(n, dtype=np.uint32)
    return st


def _run(met, state, t, dt, nsteps, mode, prm=None, seed=0, step0=0, windows=None):
    st = copy_state(state)
    for n in range(nsteps):
        t_n = t + n * dt
        sel = _windows_active(st, t_n, windows)
        lon, lat, p = st["lon"][sel], st["lat"][sel], st["p"][sel]
        if mode == "advect":
            lon, lat, p, _ = _midpoint(met, lon, lat, p, t_n, dt, sigma=False)
        elif mode == "diffuse":
            s2 = met.wind(lon, lat, p, t_n, sigma=True)[3:]
            lon, lat, p = _diffusion(met, st, sel, lon, lat, p, s2, step0 + n, seed, dt, prm)
        else:  # fused step
            lon, lat, p, s2 = _midpoint(met, lon, lat, p, t_n, dt, sigma=True)
            lon, lat, p = _diffusion(met, st, sel, lon, lat, p, s2, step0 + n, seed, dt, prm)
        lon, lat, p = position_bc(lon, lat, p, met.lon0, met.pmin, met.pmax)
        st["lon"][sel], st["lat"][sel], st["p"][sel] = lon, lat, p
    return st


def advect(met, state, t, dt, nsteps, windows=None):
    """``nsteps`` midpoint advection steps from time t (each followed by the BCs)."""
    return _run(met, state, t, dt, nsteps, "advect", windows=windows)


def diffuse(met, state, t, dt, prm, seed, step0, nsteps, windows=None):
    """Diffusion only: subgrid variance and displacement at the current position."""
    return _run(met, state, t, dt, nsteps, "diffuse", prm, seed, step0, windows)


def step(met, state, t, dt, prm, seed, step0, nsteps, windows=None):
    """Fused advection + turbulent + mesoscale diffusion + BCs."""
    return _run(met, state, t, dt, nsteps, "step", prm, seed, step0, windows)
