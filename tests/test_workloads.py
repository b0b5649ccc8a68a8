"""The synthetic inputs follow their stated recipe (no GPU): grids, the analytic 2-degree
wind, the Fourier-mode fields (rms, omega profile, 24-hour period, cos(lat) factor at the
poles), uniform particles and column releases."""
import numpy as np
import pytest

from workloads import (cfg1_snapshot, column_releases, fourier_modes, fourier_snapshot, grid_2deg_20lev,
                       grid_global, uniform_particles)
from workloads.fields import DAY, P0, grid_03deg_137lev, grid_1deg_60lev


def test_grids():
    for g, (nx, ny, nz, ptop) in ((grid_2deg_20lev(), (180, 91, 20, 1e3)), (grid_1deg_60lev(), (360, 181, 60, 1e3)),
                                  (grid_03deg_137lev(), (1200, 601, 137, 1.0))):
        assert (g.nx, g.ny, g.nz) == (nx, ny, nz)
        assert g.nx * g.dlon == pytest.approx(360.0) and g.lons[0] == 0.0
        assert g.lats[0] == -90.0 and g.lats[-1] == pytest.approx(90.0)
        assert g.plev[0] == 1e5 and g.plev[-1] == pytest.approx(ptop)
        assert np.all(np.diff(g.plev) < 0)
        r = np.log(g.plev[1:] / g.plev[:-1])
        np.testing.assert_allclose(r, r[0])                    # log-spaced


def test_cfg1_analytic_wind_at_the_nodes():
    g = grid_2deg_20lev()
    s = cfg1_snapshot(g)
    lat = np.radians(g.lats)[None, :, None]
    lon = np.radians(g.lons)[None, None, :]
    u = 40.0 * np.cos(lat) + 30.0 * np.exp(-((np.degrees(lat) - 45.0) / 10.0) ** 2)
    np.testing.assert_allclose(s["u"], np.broadcast_to(u, s["u"].shape), rtol=1e-6, atol=1e-5)
    assert np.all(s["v"] == 0)
    np.testing.assert_allclose(s["w"], np.broadcast_to(0.05 * np.sin(2 * lon) * np.cos(lat), s["w"].shape),
                               atol=1e-8)


@pytest.mark.parametrize("multiscale", [False, True])
def test_fourier_fields_follow_the_recipe(multiscale):
    g = grid_global(72, 37, 12)
    m = fourier_modes(3, multiscale=multiscale, with_T=True)
    f0 = fourier_snapshot(g, m, 0.0)
    for k in ("u", "v"):
        assert np.sqrt(np.mean(f0[k].astype(np.float64) ** 2)) == pytest.approx(20.0, rel=1e-5)
        np.testing.assert_allclose(f0[k][:, [0, -1], :], 0.0, atol=1e-4)    # cos(lat) factor at the poles
    w = f0["w"].astype(np.float64)
    assert np.sqrt(np.mean(w[0] ** 2)) == pytest.approx(0.5, rel=1e-5)       # lowest level
    T = f0["T"].astype(np.float64)
    assert np.mean(T) == pytest.approx(250.0, abs=2.0)
    assert np.sqrt(np.mean((T - 250.0) ** 2)) == pytest.approx(15.0, rel=1e-4)
    # integer cycles per day: 24-hour periodic, and different within the day
    f1 = fourier_snapshot(g, m, DAY)
    for k in ("u", "v", "w", "T"):
        np.testing.assert_allclose(f1[k], f0[k], rtol=1e-5, atol=1e-5 * np.abs(f0[k]).max())
    f6 = fourier_snapshot(g, m, DAY / 4)
    assert np.abs(f6["u"] - f0["u"]).max() > 1.0


def test_omega_profile_scales_with_pressure():
    """omega is one field shape times p/p0 per level (rescaled at the lowest level), so with
    no vertical phase (q = 0 for every mode) the levels are exact multiples of level 0."""
    g = grid_global(36, 19, 8)
    m = fourier_modes(4)
    m.comps["w"].q[:] = 0
    w = fourier_snapshot(g, m, 0.0)["w"].astype(np.float64)
    for k in range(g.nz):
        np.testing.assert_allclose(w[k], w[0] * g.plev[k] / g.plev[0], rtol=1e-5, atol=1e-9)
    assert P0 == 1e5


def test_uniform_particles():
    g = grid_1deg_60lev()
    st = uniform_particles(200_000, g.plev, seed=5, lat_max=80.0, id0=7)
    assert st["lon"].min() >= 0.0 and st["lon"].max() < 360.0
    assert np.abs(st["lat"]).max() <= 80.0
    assert st["p"].min() >= g.plev[-1] and st["p"].max() <= g.plev[0]
    lnp = np.log(st["p"])
    assert np.mean(lnp) == pytest.approx(0.5 * (np.log(g.plev[0]) + np.log(g.plev[-1])), abs=0.02)
    np.testing.assert_array_equal(st["id"], np.arange(200_000, dtype=np.uint32) + 7)
    assert np.all(st["release"] == 0)
    again = uniform_particles(200_000, g.plev, seed=5, lat_max=80.0, id0=7)
    for k in st:
        np.testing.assert_array_equal(st[k], again[k])          # seeded


def test_column_releases():
    rel = column_releases(64, seed=4)
    assert np.all(rel.t_start == 0)
    assert rel.t_end.min() >= 6 * 3600.0 and rel.t_end.max() <= 72 * 3600.0
    assert rel.counts.min() >= 1e3 and rel.counts.max() <= 1e6
    st = rel.particles
    n = int(rel.counts.sum())
    assert st["lon"].size == n and np.array_equal(st["id"], np.arange(n, dtype=np.uint32))
    z = -7000.0 * np.log(st["p"] / 101325.0)
    assert z.min() >= 1000.0 - 1e-6 and z.max() <= 20000.0 + 1e-6
    for r in (0, 17, 63):
        sel = st["release"] == r
        assert sel.sum() == rel.counts[r]
        assert np.unique(st["lon"][sel]).size == 1 and np.unique(st["lat"][sel]).size == 1


def test_initial_weights_are_the_oracle_init():
    """The network's seeded starting point equals the oracle's own draw (same order, same rule)."""
    from oracle import surrogate as S
    from workloads import initial_weights
    for seed in (0, 5):
        np.testing.assert_array_equal(initial_weights(seed), S.flatten(S.init_params(seed)).astype(np.float32))
