"""Pins of the oracle's 4D linear interpolation."""
import numpy as np

from oracle import interp
from oracle.transport import Met
from workloads import grid_global, grid_2deg_20lev


def _trilinear_field(grid, coef):
    """A field that is trilinear in (lon, lat, p): exactly reproduced inside each cell."""
    a, b, c, d, e, f, g, h = coef
    lon = grid.lons[None, None, :]
    lat = grid.lats[None, :, None]
    p = grid.plev[:, None, None]
    return a + b * lon + c * lat + d * p + e * lon * lat + f * lon * p + g * lat * p + h * lon * lat * p


def _ftrue(coef, lon, lat, p):
    a, b, c, d, e, f, g, h = coef
    return a + b * lon + c * lat + d * p + e * lon * lat + f * lon * p + g * lat * p + h * lon * lat * p


def test_trilinear_fields_reproduced_exactly():
    grid = grid_2deg_20lev()
    rng = np.random.default_rng(0)
    coef = rng.standard_normal(8) * np.array([1, 0.1, 0.1, 1e-5, 1e-3, 1e-6, 1e-6, 1e-8])
    fld = _trilinear_field(grid, coef)
    n = 5000
    lon = rng.uniform(0.0, 357.9, n)          # keep the cell away from the periodic seam
    lat = rng.uniform(-90, 90, n)
    p = np.exp(rng.uniform(np.log(grid.plev[-1]), np.log(grid.plev[0]), n))
    loc = interp.locate(grid, lon, lat, p)
    got = interp.trilinear(fld, loc)
    np.testing.assert_allclose(got, _ftrue(coef, lon, lat, p), rtol=1e-11, atol=1e-11)


def test_time_interpolation_linear():
    grid = grid_2deg_20lev()
    rng = np.random.default_rng(1)
    c0 = rng.standard_normal(8) * 0.01
    c1 = rng.standard_normal(8) * 0.01
    f0 = {k: _trilinear_field(grid, c0) for k in ("u", "v", "w")}
    f1 = {k: _trilinear_field(grid, c1) for k in ("u", "v", "w")}
    m = Met(grid, 0.0, f0, 21600.0, f1)
    lon, lat, p = np.array([10.3, 200.1]), np.array([-33.0, 71.7]), np.array([50000.0, 2345.0])
    for t in (0.0, 5000.0, 21600.0):
        w = t / 21600.0
        u, _, _ = m.wind(lon, lat, p, t)
        np.testing.assert_allclose(u, (1 - w) * _ftrue(c0, lon, lat, p) + w * _ftrue(c1, lon, lat, p),
                                   rtol=1e-11, atol=1e-12)


def test_brute_force_tiny_grid():
    """Independent sum over the 8 corners with explicit weights on a 4 x 3 x 3 grid."""
    grid = grid_global(4, 3, 3, 1e5, 5e4)
    rng = np.random.default_rng(2)
    f = rng.standard_normal((3, 3, 4))
    for _ in range(200):
        lon, lat = rng.uniform(-400, 800), rng.uniform(-90, 90)
        p = rng.uniform(4e4, 1.1e5)
        got = interp.trilinear(f, interp.locate(grid, np.array([lon]), np.array([lat]), np.array([p])))[0]
        # brute force: walk the nodes, weights from distances
        x = ((lon % 360.0) / 90.0)
        i0 = int(np.floor(x)) % 4
        fx = x - np.floor(x)
        y = (lat + 90.0) / 90.0
        j0 = min(int(np.floor(y)), 1)
        fy = y - j0
        pc = min(max(p, grid.plev[-1]), grid.plev[0])
        k0 = 0 if pc >= grid.plev[1] else 1
        fz = (grid.plev[k0] - pc) / (grid.plev[k0] - grid.plev[k0 + 1])
        ref = 0.0
        for dk, wk in ((0, 1 - fz), (1, fz)):
            for dj, wj in ((0, 1 - fy), (1, fy)):
                for di, wi in ((0, 1 - fx), (1, fx)):
                    ref += wk * wj * wi * f[k0 + dk, j0 + dj, (i0 + di) % 4]
        assert abs(got - ref) < 1e-12


def test_periodic_seam_and_shift():
    grid = grid_2deg_20lev()
    rng = np.random.default_rng(3)
    f = rng.standard_normal((grid.nz, grid.ny, grid.nx))
    fs = np.roll(f, -grid.nx // 2, axis=2)     # fs at node i = f at node i + 90 (180 degrees)
    n = 1000
    lon = rng.uniform(0, 360, n)
    lat = rng.uniform(-89, 89, n)
    p = rng.uniform(2000, 90000, n)
    a = interp.trilinear(f, interp.locate(grid, lon + 180.0, lat, p))
    b = interp.trilinear(fs, interp.locate(grid, lon, lat, p))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    # the last cell joins node nx-1 to node 0
    lon = np.array([359.0, -1.0, 719.0])
    loc = interp.locate(grid, lon, np.array([0.0] * 3), np.array([5e4] * 3))
    v = interp.trilinear(f, loc)
    assert np.all(loc[0] == grid.nx - 1) and np.all(loc[1] == 0)
    np.testing.assert_allclose(v, v[0], rtol=1e-12)


def test_pressure_clamp_and_nodes():
    grid = grid_2deg_20lev()
    f = np.broadcast_to(grid.plev[:, None, None], (grid.nz, grid.ny, grid.nx)).copy()
    p = np.array([2e5, grid.plev[0], grid.plev[7], 0.5 * (grid.plev[3] + grid.plev[4]), grid.plev[-1], 1.0])
    loc = interp.locate(grid, np.zeros(6), np.zeros(6), p)
    got = interp.trilinear(f, loc)
    np.testing.assert_allclose(got, np.clip(p, grid.plev[-1], grid.plev[0]), rtol=1e-13)
    # node hit exactly: zero fraction
    assert loc[6][2] == 0.0 and loc[3][2] == 7


def test_corner_variance():
    grid = grid_global(8, 5, 4)
    const = np.full((4, 5, 8), 3.0)
    loc = interp.locate(grid, np.array([17.0]), np.array([10.0]), np.array([60000.0]))
    assert interp.corner_variance(const, loc)[0] == 0.0
    # checkerboard +-A along longitude: w-weighted spread = 4 A^2 fx (1 - fx)
    A = 2.5
    chk = np.fromfunction(lambda k, j, i: np.where(i % 2 == 0, A, -A), (4, 5, 8))
    for lon in (45.0, 50.0, 60.0, 67.5, 89.0):
        loc = interp.locate(grid, np.array([lon]), np.array([10.0]), np.array([60000.0]))
        fx = loc[4][0]
        assert abs(interp.corner_variance(chk, loc)[0] - 4 * A * A * fx * (1 - fx)) < 1e-12


def test_corner_variance_continuous_across_faces():
    """Both cells sharing a face give the same variance on it."""
    grid = grid_2deg_20lev()
    rng = np.random.default_rng(7)
    f = rng.standard_normal((grid.nz, grid.ny, grid.nx))
    eps = 1e-9
    lat = rng.uniform(-80, 80, 200)
    p = rng.uniform(2e3, 9e4, 200)
    face_lon = 2.0 * rng.integers(1, 170, 200)
    a = interp.corner_variance(f, interp.locate(grid, face_lon - eps, lat, p))
    b = interp.corner_variance(f, interp.locate(grid, face_lon + eps, lat, p))
    np.testing.assert_allclose(a, b, atol=1e-6)
    face_lat = -80.0 + 2.0 * rng.integers(1, 79, 200)
    lon = rng.uniform(0, 358, 200)
    a = interp.corner_variance(f, interp.locate(grid, lon, face_lat - eps, p))
    b = interp.corner_variance(f, interp.locate(grid, lon, face_lat + eps, p))
    np.testing.assert_allclose(a, b, atol=1e-6)
    # brute force at one point: weighted spread about the weighted mean
    loc = interp.locate(grid, np.array([33.3]), np.array([-12.7]), np.array([41234.0]))
    w = interp.corner_weights(loc)[:, 0]
    c = interp.corners(f, loc)[:, 0]
    assert abs(w.sum() - 1) < 1e-15
    m = sum(wi * ci for wi, ci in zip(w, c))
    ref = sum(wi * (ci - m) ** 2 for wi, ci in zip(w, c))
    assert abs(interp.corner_variance(f, loc)[0] - ref) < 1e-13
