"""Pins of the oracle's cell-key sort."""
import numpy as np

from oracle import sort as osort
from workloads import grid_2deg_20lev, uniform_particles


def test_hand_keys():
    grid = grid_2deg_20lev()   # 180 x 91 x 20, dlon = dlat = 2
    # lon 3.0 -> i = 1; lat -87.0 -> y = 1.5 -> j = 1; p = plev[5] exactly -> k = 5
    # lon 359.5 -> i = 179; lat 90 -> j = 89 (clamped); p = 1e5 -> k = 0
    # lon 0.0 -> i = 0; lat -90 -> j = 0; p = 1000 (top) -> k = 18 (clamped)
    lon = np.array([3.0, 359.5, 0.0])
    lat = np.array([-87.0, 90.0, -90.0])
    p = np.array([grid.plev[5], 1e5, 1e3])
    keys = osort.cell_keys(grid, lon, lat, p)
    expect = [(1 * 180 + 1) * 20 + 5, (89 * 180 + 179) * 20 + 0, (0 * 180 + 0) * 20 + 18]
    np.testing.assert_array_equal(keys, expect)


def test_sorted_stable_permutation():
    grid = grid_2deg_20lev()
    st = uniform_particles(5000, grid.plev, seed=3)
    # force many equal keys: snap a third of the particles onto one point
    st["lon"][::3], st["lat"][::3], st["p"][::3] = 41.0, 12.0, 50000.0
    perm = osort.sort_permutation(grid, st)
    assert np.array_equal(np.sort(perm), np.arange(5000))
    keys = osort.cell_keys(grid, st["lon"], st["lat"], st["p"])[perm]
    assert np.all(np.diff(keys.astype(np.int64)) >= 0)
    # stability: within equal keys the original index increases
    same = np.diff(keys.astype(np.int64)) == 0
    assert np.all(np.diff(perm)[same] > 0)
    out = osort.sort_state(grid, st)
    np.testing.assert_array_equal(out["id"], st["id"][perm])


def test_inactive_releases_sorted_last_in_order():
    grid = grid_2deg_20lev()
    st = uniform_particles(12, grid.plev, seed=5)
    st["release"] = np.array([0, 1, 2, 0, 1, 2, 5, 0, 1, 2, 0, 1], np.uint32)
    ts = np.array([0.0, 100.0, 0.0])
    te = np.array([50.0, 200.0, 1e9])
    # at t = 60: release 0 ended, release 1 not started, release 2 active, 5 unknown
    perm = osort.sort_permutation_at(grid, st, 60.0, (ts, te))
    active = np.flatnonzero(st["release"] == 2)
    inactive = np.flatnonzero(st["release"] != 2)
    keys = osort.cell_keys(grid, st["lon"], st["lat"], st["p"])
    np.testing.assert_array_equal(perm[:active.size], active[np.argsort(keys[active], kind="stable")])
    np.testing.assert_array_equal(perm[active.size:], inactive)
    # without windows the rule reduces to the plain sort when everything is active
    all_on = (np.zeros(6), np.full(6, 1e9))
    st["release"][:] = 0
    np.testing.assert_array_equal(osort.sort_permutation_at(grid, st, 5.0, all_on),
                                  osort.sort_permutation(grid, st))
