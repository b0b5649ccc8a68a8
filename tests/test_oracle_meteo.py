"""Pins of the oracle's met sampling and particle gridding."""
import numpy as np

from oracle import meteo
from workloads import grid_global, uniform_particles


def test_sample_reproduces_trilinear_field_and_time_lerp():
    grid = grid_global(24, 13, 8)
    lon = grid.lons[None, None, :]
    lat = grid.lats[None, :, None]
    p = grid.plev[:, None, None]
    f0 = {"u": 1.0 + 0.01 * lon + 0 * lat + 0 * p, "v": 0.1 * lat + 0 * lon + 0 * p,
          "w": 1e-5 * p + 0 * lon + 0 * lat, "T": 200.0 + 0.5 * lat + 1e-4 * p + 0 * lon}
    f1 = {k: 2 * v for k, v in f0.items()}
    rng = np.random.default_rng(0)
    n = 500
    lo, la = rng.uniform(0, 344, n), rng.uniform(-90, 90, n)
    pp = np.exp(rng.uniform(np.log(grid.plev[-1]), np.log(grid.plev[0]), n))
    s = meteo.sample(grid, f0, 0.0, f1, 100.0, 25.0, lo, la, pp)
    scale = 1.25
    np.testing.assert_allclose(s["u"], scale * (1.0 + 0.01 * lo), rtol=1e-12)
    np.testing.assert_allclose(s["v"], scale * 0.1 * la, atol=1e-12)
    np.testing.assert_allclose(s["T"], scale * (200.0 + 0.5 * la + 1e-4 * pp), rtol=1e-12)


def test_grid_counts_sum_and_hand_cells():
    grid = grid_global(36, 19, 10)
    st = uniform_particles(10_000, grid.plev, seed=4)
    c = meteo.grid_counts(grid, st["lon"], st["lat"], st["p"])
    assert c.sum() == 10_000 and c.size == 36 * 19 * 10
    # three particles in one known cell: lon 15 (i=1), lat -75 (y=1.5 -> j=1), p = level 3 exactly (k=3)
    lon = np.array([15.0, 16.0, 19.0])
    lat = np.array([-75.0, -74.0, -71.0])
    p = np.full(3, grid.plev[3])
    c = meteo.grid_counts(grid, lon, lat, p)
    key = (1 * 36 + 1) * 10 + 3
    assert c[key] == 3 and c.sum() == 3
