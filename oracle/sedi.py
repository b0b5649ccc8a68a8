"""Sedimentation -- TEST INFRASTRUCTURE ONLY.

``module_sedi`` (Section 3.2) moves particles along the trajectory by
sedimentation; the paper gives no formula.  The reading used: spherical
particles of radius r and density rho_p settle at the Stokes terminal velocity
with the Cunningham slip correction,

    v_s = 2 r^2 (rho_p - rho_air) g C / (9 eta),
    C   = 1 + Kn (1.257 + 0.4 exp(-1.1 / Kn)),  Kn = lambda / r,
    lambda = 2 eta / (rho_air * vbar),  vbar = sqrt(8 R_d T / pi),
    eta = 1.8325e-5 (416.16 / (T + 120)) (T / 296.16)^1.5   (Sutherland),
    rho_air = p / (R_d T),

with T interpolated at the particle, and the fall becomes a pressure increase
dp = rho_air g v_s dt per step (p clamped to the level range).
"""
from __future__ import annotations

import numpy as np

from . import interp

G = 9.80665
R_D = 287.058


def viscosity(T):
    T = np.asarray(T, np.float64)
    return 1.8325e-5 * (416.16 / (T + 120.0)) * (T / 296.16) ** 1.5


def settling_velocity(p, T, r, rho_p):
    p, T, r, rho_p = (np.asarray(a, np.float64) for a in (p, T, r, rho_p))
    rho = p / (R_D * T)
    eta = viscosity(T)
    vbar = np.sqrt(8.0 * R_D * T / np.pi)
    lam = 2.0 * eta / (rho * vbar)
    kn = lam / r
    cc = 1.0 + kn * (1.257 + 0.4 * np.exp(-1.1 / kn))
    return 2.0 * r * r * (rho_p - rho) * G * cc / (9.0 * eta)


def sediment(grid, T0, t0, T1, t1, state, r, rho_p, t, dt, nsteps):
    """nsteps sedimentation steps from time t; returns the new pressures."""
    p = np.array(state["p"], dtype=np.float64, copy=True)
    lon, lat = np.asarray(state["lon"], np.float64), np.asarray(state["lat"], np.float64)
    pmin, pmax = float(np.min(grid.plev)), float(np.max(grid.plev))
    for n in range(nsteps):
        tn = t + n * dt
        loc = interp.locate(grid, lon, lat, p)
        w = interp.time_weight(tn, t0, t1)
        T = (1 - w) * interp.trilinear(np.asarray(T0, np.float64), loc) + w * interp.trilinear(
            np.asarray(T1, np.float64), loc)
        vs = settling_velocity(p, T, r, rho_p)
        p = np.clip(p + p / (R_D * T) * G * vs * dt, pmin, pmax)
    return p
