"""Grid descriptions and seeded synthetic met snapshots (inputs only).

The paper reads gridded meteorological data (winds u, v, omega and more) from
netCDF files in ``read_met`` (Section 3.1) and carries two snapshots ``met0`` and
``met1`` bracketing the model time (Section 4.1, data regions).  No such data is
available here, so this module synthesises snapshots on regular longitude x
latitude x pressure grids:

* ``cfg1_snapshot`` -- the steady analytic wind of the 2 degree / 20 level case:
  u = 40 cos(phi) + 30 exp(-((phi - 45)/10)^2) m/s, v = 0,
  omega = 0.05 sin(2 lambda) cos(phi) Pa/s, sampled at the grid nodes.
* ``fourier_snapshot`` -- a seeded sum of Fourier modes on the sphere
  A cos(phi) cos(m lambda + 2 n phi + q ln(p/p0) + 2 pi h t / 24 h + phase),
  each component rescaled to a prescribed grid-point rms.  Integer ``h`` makes
  the field 24 h periodic, so four snapshots 6 h apart cover a day and longer
  runs cycle them.  The cos(phi) factor keeps u / (R cos phi) finite at the
  poles.  The sum is evaluated separably (a contraction over the mode indices),
  which is exact and fast even on the 0.3 degree grid.

Arrays are returned as float32 with layout ``[level][lat][lon]`` (C order),
the layout in which met data are handed to the library.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

P0 = 100000.0          # reference pressure of the mode phase and omega profile [Pa]
DAY = 86400.0


@dataclass
class Grid:
    """Regular global lon-lat grid with ``nz`` pressure levels.

    ``plev`` is in Pa and strictly decreasing (level 0 is the lowest level).
    Longitude is periodic: ``nx * dlon == 360``.
    """
    nx: int
    ny: int
    nz: int
    lon0: float
    dlon: float
    lat0: float
    dlat: float
    plev: np.ndarray = field(repr=False)

    @property
    def lons(self) -> np.ndarray:
        return self.lon0 + self.dlon * np.arange(self.nx, dtype=np.float64)

    @property
    def lats(self) -> np.ndarray:
        return self.lat0 + self.dlat * np.arange(self.ny, dtype=np.float64)

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nz


def log_levels(p_bot: float, p_top: float, nz: int) -> np.ndarray:
    """Pressure levels log-spaced from ``p_bot`` down to ``p_top`` [Pa]."""
    k = np.arange(nz, dtype=np.float64)
    return p_bot * (p_top / p_bot) ** (k / (nz - 1))


def grid_global(nx: int, ny: int, nz: int, p_bot: float = 1e5, p_top: float = 1e3) -> Grid:
    """Global grid: lon 0 .. 360-dlon, lat -90 .. 90 inclusive."""
    return Grid(nx, ny, nz, 0.0, 360.0 / nx, -90.0, 180.0 / (ny - 1),
                log_levels(p_bot, p_top, nz))


def grid_2deg_20lev() -> Grid:
    """2 degree global grid (180 x 91) with 20 levels, 1000 -> 10 hPa."""
    return grid_global(180, 91, 20, 1e5, 1e3)


def grid_1deg_60lev() -> Grid:
    """1 degree global grid (360 x 181) with 60 levels, 1000 -> 10 hPa."""
    return grid_global(360, 181, 60, 1e5, 1e3)


def grid_03deg_137lev() -> Grid:
    """0.3 degree global grid (1200 x 601) with 137 levels, 1000 -> 0.01 hPa."""
    return grid_global(1200, 601, 137, 1e5, 1.0)


# --------------------------------------------------------------------------
# 2 degree analytic case
# --------------------------------------------------------------------------

def cfg1_analytic_wind(lon_deg, lat_deg, p_pa):
    """The analytic steady wind of the 2 degree case at arbitrary points.

    Returns (u [m/s], v [m/s], omega [Pa/s]) as float64 numpy arrays.  The
    pressure argument is unused (the wind has no vertical structure) but kept
    so the signature matches any wind callable.
    """
    lam = np.radians(np.asarray(lon_deg, dtype=np.float64))
    phi_deg = np.asarray(lat_deg, dtype=np.float64)
    phi = np.radians(phi_deg)
    u = 40.0 * np.cos(phi) + 30.0 * np.exp(-((phi_deg - 45.0) / 10.0) ** 2)
    v = np.zeros_like(u)
    w = 0.05 * np.sin(2.0 * lam) * np.cos(phi)
    shape = np.broadcast(lam, phi, np.asarray(p_pa)).shape
    return (np.broadcast_to(u, shape).copy(), np.broadcast_to(v, shape).copy(),
            np.broadcast_to(w, shape).copy())


def cfg1_snapshot(grid: Grid) -> dict:
    """Analytic wind sampled at the grid nodes: dict u, v, w -> float32 [nz][ny][nx]."""
    lon = grid.lons[None, None, :]
    lat = grid.lats[None, :, None]
    p = grid.plev[:, None, None]
    u, v, w = cfg1_analytic_wind(lon, lat, p)
    shape = (grid.nz, grid.ny, grid.nx)
    return {k: np.ascontiguousarray(np.broadcast_to(a, shape), dtype=np.float32)
            for k, a in (("u", u), ("v", v), ("w", w))}


# --------------------------------------------------------------------------
# Seeded Fourier modes on the sphere
# --------------------------------------------------------------------------

@dataclass
class ModeSet:
    """Mode parameters of one field component."""
    m: np.ndarray        # zonal wavenumber
    n: np.ndarray        # meridional index (phase 2 n phi)
    q: np.ndarray        # vertical index (phase q ln(p/p0))
    h: np.ndarray        # cycles per day
    phase: np.ndarray    # radians
    amp: np.ndarray      # relative amplitude (rescaled to the target rms)


@dataclass
class FourierModes:
    comps: dict          # name -> ModeSet
    rms: dict            # name -> target grid-point rms
    offset: dict         # name -> constant added after scaling


def _draw_modes(rng, n_modes, m_max, n_max, q_max, h_max, slope):
    m = rng.integers(1, m_max + 1, n_modes)
    n = rng.integers(0, n_max + 1, n_modes)
    q = rng.integers(0, q_max + 1, n_modes)
    h = rng.integers(0, h_max + 1, n_modes)
    phase = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    amp = rng.uniform(0.5, 1.0, n_modes)
    if slope is not None:
        k = np.sqrt(m.astype(np.float64) ** 2 + (2.0 * n) ** 2)
        amp = amp * k ** slope
    return ModeSet(m, n, q, h, phase, amp)


def fourier_modes(seed: int, n_modes: int = 64, multiscale: bool = False,
                  with_T: bool = False) -> FourierModes:
    """Draw the mode parameters of u, v, omega (and T) from ``seed``.

    Smooth case: m in 1..8, n in 0..4, q in 0..3, h in 0..2.
    Multiscale case: m in 1..180, n in 0..90, amplitude ~ k^(-5/6)
    (energy spectrum ~ k^(-5/3)).
    Target rms: 20 m/s for u and v at every level; omega 0.5 Pa/s rms at the
    lowest level with a p/p0 profile; T 15 K around 250 K.
    """
    rng = np.random.default_rng(seed)
    names = ["u", "v", "w"] + (["T"] if with_T else [])
    comps = {}
    for name in names:
        if multiscale:
            comps[name] = _draw_modes(rng, n_modes, 180, 90, 3, 2, -5.0 / 6.0)
        else:
            comps[name] = _draw_modes(rng, n_modes, 8, 4, 3, 2, None)
    rms = {"u": 20.0, "v": 20.0, "w": 0.5, "T": 15.0}
    offset = {"u": 0.0, "v": 0.0, "w": 0.0, "T": 250.0}
    return FourierModes(comps, {k: rms[k] for k in names}, {k: offset[k] for k in names})


def _synth(grid: Grid, ms: ModeSet, t: float, device) -> torch.Tensor:
    """Separable evaluation of sum_modes amp cos(m lam + 2 n phi + q ln(p/p0) + 2 pi h t/day + phase).

    Returns float64 [nz][ny][nx] on ``device`` (without the cos(phi) factor).
    """
    M, N, Q = int(ms.m.max()) + 1, int(ms.n.max()) + 1, int(ms.q.max()) + 1
    coef = np.zeros((M, N, Q), dtype=np.complex128)
    ang = ms.phase + 2.0 * math.pi * ms.h * (t / DAY)
    np.add.at(coef, (ms.m, ms.n, ms.q), ms.amp * np.exp(1j * ang))
    C = torch.from_numpy(coef).to(device)
    lam = torch.from_numpy(np.radians(grid.lons)).to(device)
    phi = torch.from_numpy(np.radians(grid.lats)).to(device)
    lnp = torch.from_numpy(np.log(grid.plev / P0)).to(device)
    X = torch.exp(1j * torch.arange(M, device=device, dtype=torch.float64)[:, None] * lam[None, :])
    Y = torch.exp(1j * 2.0 * torch.arange(N, device=device, dtype=torch.float64)[:, None] * phi[None, :])
    Z = torch.exp(1j * torch.arange(Q, device=device, dtype=torch.float64)[:, None] * lnp[None, :])
    F = torch.einsum("mnq,mx->nqx", C, X)              # (N, Q, nx)
    G = torch.einsum("nqx,ny->qyx", F, Y)              # (Q, ny, nx)
    out = torch.matmul(Z.transpose(0, 1), G.reshape(Q, -1)).real  # (nz, ny*nx)
    return out.reshape(grid.nz, grid.ny, grid.nx)


def fourier_snapshot(grid: Grid, modes: FourierModes, t: float, device="cpu",
                     as_numpy: bool = True):
    """Snapshot at time ``t`` [s]: dict name -> float32 [nz][ny][nx].

    The rescaling factor of each component is taken from its t = 0 field on the
    same grid, so every snapshot of a run uses the same factor.
    """
    device = torch.device(device)
    cosphi = torch.from_numpy(np.cos(np.radians(grid.lats))).to(device)[None, :, None]
    prof_w = torch.from_numpy(grid.plev / P0).to(device)[:, None, None]
    out = {}
    for name, ms in modes.comps.items():
        raw0 = _synth(grid, ms, 0.0, device) * cosphi
        raw = raw0 if t == 0.0 else _synth(grid, ms, t, device) * cosphi
        if name == "w":
            base = torch.sqrt(torch.mean(raw0[0] ** 2))
            val = raw * (modes.rms[name] / base) * prof_w / prof_w[0]
        else:
            base = torch.sqrt(torch.mean(raw0 ** 2))
            val = raw * (modes.rms[name] / base) + modes.offset[name]
        val = val.to(torch.float32).contiguous()
        out[name] = val.cpu().numpy() if as_numpy else val
    return out
