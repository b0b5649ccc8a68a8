"""Pins of the oracle's trajectory stepping: closed forms, moments, boundary cases."""
import numpy as np
import pytest

from oracle import transport as tr
from oracle.errors import lon_diff
from workloads import grid_2deg_20lev, cfg1_analytic_wind, cfg1_snapshot

R = tr.R_EARTH
DEG = 180.0 / np.pi


def _const_met(grid, u=0.0, v=0.0, w=0.0, t1=21600.0):
    shape = (grid.nz, grid.ny, grid.nx)
    f = {"u": np.full(shape, u), "v": np.full(shape, v), "w": np.full(shape, w)}
    return tr.Met(grid, 0.0, f, t1, f)


def _state(lon, lat, p):
    n = len(lon)
    return {"lon": np.asarray(lon, float), "lat": np.asarray(lat, float), "p": np.asarray(p, float),
            "id": np.arange(n, dtype=np.uint32), "release": np.zeros(n, np.uint32)}


def test_constant_zonal_wind_shift():
    """Constant u, v = omega = 0: every step moves lon by u dt / (R cos(lat)) * 180/pi."""
    grid = grid_2deg_20lev()
    u, dt, n = 17.0, 180.0, 120
    met = _const_met(grid, u=u)
    lat = np.array([-75.0, -30.0, 0.0, 12.5, 60.0, 80.0])
    lon0 = np.array([0.0, 100.0, 359.9, 200.0, 45.0, 300.0])
    st = tr.advect(met, _state(lon0, lat, np.full(6, 50000.0)), 0.0, dt, n)
    expect = lon0 + n * u * dt / (R * np.cos(np.radians(lat))) * DEG
    np.testing.assert_allclose(lon_diff(st["lon"], expect), 0.0, atol=1e-9)
    np.testing.assert_array_equal(st["lat"], lat)
    np.testing.assert_array_equal(st["p"], 50000.0)


def test_solid_body_rotation_returns_after_one_period():
    """u = 40 cos(lat): d lon/dt = 40/R for every latitude; period 2 pi R / 40."""
    period = 2 * np.pi * R / 40.0
    nsteps = 5560
    dt = period / nsteps

    def wind(lon, lat, p, t):
        c = np.cos(np.radians(lat))
        return 40.0 * c, 0.0 * c, 0.0 * c

    met = tr.AnalyticMet(wind, 0.0, period, 1e3, 1e5)
    rng = np.random.default_rng(0)
    lon0, lat0 = rng.uniform(0, 360, 200), rng.uniform(-80, 80, 200)
    st = tr.advect(met, _state(lon0, lat0, np.full(200, 5e4)), 0.0, dt, nsteps)
    assert np.max(np.abs(lon_diff(st["lon"], lon0))) < 1e-8
    # half a period: opposite meridian
    st = tr.advect(met, _state(lon0, lat0, np.full(200, 5e4)), 0.0, dt, nsteps // 2)
    assert np.max(np.abs(lon_diff(st["lon"], lon0 + 180.0))) < 1e-8


def test_uniform_omega_linear_pressure_drift():
    grid = grid_2deg_20lev()
    w, dt, n = -0.7, 180.0, 100
    met = _const_met(grid, w=w)
    p0 = np.array([90000.0, 40000.0, 20000.0])
    st = tr.advect(met, _state([1.0, 2.0, 3.0], [0.0, 10.0, -10.0], p0), 0.0, dt, n)
    np.testing.assert_allclose(st["p"], p0 + w * n * dt, rtol=1e-14)
    # until the clamp at the top level
    st = tr.advect(met, _state([1.0], [0.0], [1500.0]), 0.0, dt, n)
    assert st["p"][0] == grid.plev[-1]


def _cfg1_exact(lon0, lat0, p0, t):
    u, _, _ = cfg1_analytic_wind(lon0, lat0, p0)
    a = u / (R * np.cos(np.radians(lat0)))              # rad/s
    l0 = np.radians(lon0)
    lon = lon0 + a * t * DEG
    p = p0 + 0.05 * np.cos(np.radians(lat0)) * (np.cos(2 * l0) - np.cos(2 * l0 + 2 * a * t)) / (2 * a)
    return lon, p


def test_cfg1_exact_orbit_and_second_order():
    """Steady analytic wind: lat fixed, lon linear in t, p in closed form; midpoint error O(dt^2)."""
    def wind(lon, lat, p, t):
        return cfg1_analytic_wind(lon, lat, p)

    met = tr.AnalyticMet(wind, 0.0, 21600.0, 1e3, 1e5)
    rng = np.random.default_rng(1)
    n = 300
    lon0, lat0 = rng.uniform(0, 360, n), rng.uniform(-80, 80, n)
    p0 = np.exp(rng.uniform(np.log(3e4), np.log(7e4), n))
    errs = []
    for dt in (360.0, 180.0, 90.0):
        nsteps = int(round(21600.0 / dt))
        st = tr.advect(met, _state(lon0, lat0, p0), 0.0, dt, nsteps)
        lon_e, p_e = _cfg1_exact(lon0, lat0, p0, 21600.0)
        np.testing.assert_array_equal(st["lat"], lat0)
        assert np.max(np.abs(lon_diff(st["lon"], lon_e))) < 1e-9
        errs.append(np.max(np.abs(st["p"] - p_e)))
    assert errs[0] > 0
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5


def test_gridded_cfg1_close_to_analytic():
    """The gridded 2 degree field differs from the analytic one by interpolation error only."""
    grid = grid_2deg_20lev()
    snap = cfg1_snapshot(grid)
    met = tr.Met(grid, 0.0, snap, 21600.0, snap)
    rng = np.random.default_rng(2)
    n = 500
    lon0, lat0 = rng.uniform(0, 360, n), rng.uniform(-80, 80, n)
    p0 = np.exp(rng.uniform(np.log(3e4), np.log(7e4), n))
    st = tr.advect(met, _state(lon0, lat0, p0), 0.0, 180.0, 120)
    lon_e, p_e = _cfg1_exact(lon0, lat0, p0, 21600.0)
    # 2 degree lerp of a jet of 10 degree width: a few tenths of a degree over 6 h
    assert np.max(np.abs(lon_diff(st["lon"], lon_e))) < 0.5
    assert np.max(np.abs(st["p"] - p_e) / p_e) < 1e-2


def test_position_bc_hand_cases():
    lon = np.array([10.0, 10.0, -1.0, 360.0, 725.0, 359.0, 200.0])
    lat = np.array([91.0, -92.5, 0.0, 0.0, 0.0, 90.0, -90.0])
    p = np.array([5e4, 5e4, 2e5, 10.0, 5e4, 5e4, 5e4])
    L, P, Q = tr.position_bc(lon, lat, p, 0.0, 1e3, 1e5)
    np.testing.assert_allclose(L, [190.0, 190.0, 359.0, 0.0, 5.0, 359.0, 200.0])
    np.testing.assert_allclose(P, [89.0, -87.5, 0.0, 0.0, 0.0, 90.0, -90.0])
    np.testing.assert_allclose(Q, [5e4, 5e4, 1e5, 1e3, 5e4, 5e4, 5e4])
    # tiny negative longitude must not round to 360
    L, _, _ = tr.position_bc(np.array([-1e-17]), np.array([0.0]), np.array([5e4]), 0.0, 1e3, 1e5)
    assert 0.0 <= L[0] < 360.0


def test_release_windows_mask():
    grid = grid_2deg_20lev()
    met = _const_met(grid, u=10.0)
    st0 = _state([0.0] * 4, [0.0] * 4, [5e4] * 4)
    st0["release"] = np.array([0, 1, 2, 3], np.uint32)
    ts = np.array([0.0, 360.0, 0.0, 900.0])
    te = np.array([1e9, 1e9, 540.0, 1e9])
    st = tr.advect(met, st0, 0.0, 180.0, 5, windows=(ts, te))   # step times 0,180,...,720
    per = 10.0 * 180.0 / R * DEG
    np.testing.assert_allclose(st["lon"], [5 * per, 3 * per, 3 * per, 0.0], rtol=1e-12)


def test_turbulent_diffusion_moments():
    grid = grid_2deg_20lev()
    met = _const_met(grid)
    n, dt, ns = 20000, 180.0, 100
    st0 = _state(np.full(n, 100.0), np.zeros(n), np.full(n, 5e4))
    prm = tr.DiffParams(meso=False)
    st = tr.diffuse(met, st0, 0.0, dt, prm, seed=11, step0=0, nsteps=ns)
    dx = np.radians(st["lon"] - 100.0) * R        # at the equator: no metric factor to first order
    dy = np.radians(st["lat"]) * R
    var_h = 2 * prm.dx * dt * ns
    for d in (dx, dy):
        assert abs(d.mean()) < 5 * np.sqrt(var_h / n)
        assert abs(d.var() / var_h - 1) < 5 * np.sqrt(2 / n)
    lnp = np.log(st["p"] / 5e4)
    var_z = 2 * prm.dz * dt * ns / prm.scale_height ** 2
    assert abs(lnp.var() / var_z - 1) < 5 * np.sqrt(2 / n)


def test_mesoscale_stationary_variance_and_autocorrelation():
    grid = grid_2deg_20lev()
    A = 3.0
    chk = np.fromfunction(lambda k, j, i: np.where(i % 2 == 0, A, -A), (grid.nz, grid.ny, grid.nx))
    zero = np.zeros_like(chk)
    f = {"u": chk, "v": zero, "w": zero}
    met = tr.Met(grid, 0.0, f, 21600.0, f)
    n, dt = 4000, 180.0
    prm = tr.DiffParams(turb=False, meso=True)
    st = _state(np.full(n, 51.0), np.full(n, 1.0), np.full(n, 5e4))
    st = tr.diffuse(met, st, 0.0, dt, prm, seed=5, step0=0, nsteps=400)
    nxt = tr.diffuse(met, st, 0.0, dt, prm, seed=5, step0=400, nsteps=1)
    r = 1 - 2 * dt / 21600.0
    target = (prm.meso_f * A) ** 2 * (1 - r ** 800)
    assert abs(st["up"].var() / target - 1) < 5 * np.sqrt(2 / n)
    assert np.all(st["vp"] == 0) and np.all(st["wp"] == 0)
    rho = np.corrcoef(st["up"], nxt["up"])[0, 1]
    assert abs(rho - r) < 0.01


def test_zero_variance_no_meso_displacement():
    grid = grid_2deg_20lev()
    met = _const_met(grid, u=0.0)
    st0 = _state([10.0, 20.0], [5.0, -5.0], [5e4, 3e4])
    st = tr.diffuse(met, st0, 0.0, 180.0, tr.DiffParams(turb=False), 3, 0, 20)
    for k in ("lon", "lat", "p"):
        np.testing.assert_array_equal(st[k], st0[k])


def test_fused_step_identities():
    """Diffusion off -> step == advect; zero wind -> step == diffuse."""
    grid = grid_2deg_20lev()
    snap = cfg1_snapshot(grid)
    met = tr.Met(grid, 0.0, snap, 21600.0, snap)
    rng = np.random.default_rng(4)
    st0 = _state(rng.uniform(0, 360, 50), rng.uniform(-80, 80, 50), rng.uniform(2e3, 9e4, 50))
    off = tr.DiffParams(turb=False, meso=False)
    a = tr.advect(met, st0, 0.0, 180.0, 7)
    b = tr.step(met, st0, 0.0, 180.0, off, 1, 0, 7)
    for k in ("lon", "lat", "p"):
        np.testing.assert_array_equal(a[k], b[k])
    met0 = _const_met(grid)
    prm = tr.DiffParams()
    c = tr.diffuse(met0, st0, 0.0, 180.0, prm, 9, 3, 7)
    d = tr.step(met0, st0, 0.0, 180.0, prm, 9, 3, 7)
    for k in ("lon", "lat", "p", "up"):
        np.testing.assert_array_equal(c[k], d[k])


def test_schedule_over_intervals_equals_one_long_run():
    """The interval driver on a time-independent field equals one fused run over the whole
    span with the global step index running on (the second interval starts at step 120):
    counters and interval boundaries add nothing of their own.  Turbulent diffusion only:
    the mesoscale memory r = 1 - 2 dt/(t1 - t0) depends on the interval length by its
    definition, so it differs between one 12 h interval and two of 6 h."""
    from oracle.driver import run_schedule
    from workloads import uniform_particles
    grid = grid_2deg_20lev()
    snap = cfg1_snapshot(grid)
    st0 = uniform_particles(300, grid.plev, seed=3, lat_max=80.0)
    st0["up"] = np.zeros(300)
    st0["vp"] = np.zeros(300)
    st0["wp"] = np.zeros(300)
    prm = tr.DiffParams(meso=False)
    a = run_schedule(grid, lambda t: snap, 21600.0, st0, 0.0, 2 * 21600.0, 180.0, prm, 9)
    met = tr.Met(grid, 0.0, snap, 2 * 21600.0, snap)
    b = tr.step(met, st0, 0.0, 180.0, prm, 9, 0, 240)
    for k in ("lon", "lat", "p"):
        np.testing.assert_allclose(a[k], b[k], rtol=0, atol=1e-9)
