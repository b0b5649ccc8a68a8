"""Sort parity: cell keys and the stable permutation are bit-identical to the oracle."""
import numpy as np
import pytest
import torch

from oracle import sort as osort
from workloads import grid_1deg_60lev, grid_2deg_20lev, uniform_particles

from _gpu_common import M, make_ctx  # noqa: F401

pytestmark = pytest.mark.gpu


def _ctx(M, grid):
    z = {k: np.zeros((grid.nz, grid.ny, grid.nx), np.float32) for k in ("u", "v", "w")}
    return make_ctx(M, grid, [z, z], [0.0, 1.0])


@pytest.mark.parametrize("n", [1, 2047, 2048, 2049, 100_000])
def test_keys_and_permutation(M, n):
    grid = grid_1deg_60lev()
    ctx = _ctx(M, grid)
    st = uniform_particles(n, grid.plev, seed=n)
    # many equal keys and exact cell faces
    st["lon"][::5] = 10.0
    st["lat"][::5] = -3.0
    st["p"][::5] = grid.plev[7]
    st["lon"][1::7] = 359.99999999999994
    st["up"] = np.arange(n, dtype=np.float32)
    parts = M.Particles.from_numpy(st)
    keys = ctx.cell_keys(parts).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(keys, osort.cell_keys(grid, st["lon"], st["lat"], st["p"]))
    ctx.sort(parts)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    ref = osort.sort_state(grid, st)
    for k in ("lon", "lat", "p", "id", "release", "up"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_sort_skips_null_arrays_and_checks_workspace(M):
    grid = grid_2deg_20lev()
    ctx = _ctx(M, grid)
    st = uniform_particles(5000, grid.plev, seed=1)
    parts = M.Particles.from_numpy(st, meso=False, release=False)
    ctx.sort(parts)
    torch.cuda.synchronize()
    ref = osort.sort_state(grid, st)
    np.testing.assert_array_equal(parts.to_numpy()["id"], ref["id"])
    small = torch.empty(100, dtype=torch.uint8, device="cuda")
    with pytest.raises(M.MptracError) as e:
        ctx.sort(parts, small)
    assert e.value.code == -5


def test_keys_next_to_cell_faces(M):
    """Positions at 0, a few ulps and 1e-15 .. 1e-3 cell widths from longitude, latitude and
    level faces (both sides): the float32 fast path with its error margins and the float64
    fallback together give exactly the float64 key of the definition."""
    grid = grid_1deg_60lev()
    ctx = _ctx(M, grid)
    rng = np.random.default_rng(42)
    rel = np.array([0.0, 1e-15, 1e-12, 1e-9, 1e-7, 3e-7, 1e-6, 3e-6, 1e-5, 3e-5, 1e-4, 3e-4, 1e-3])
    rel = np.concatenate([rel, -rel[1:]])
    m = 4000
    st = uniform_particles(m * 3, grid.plev, seed=5)
    lon, lat, p = st["lon"], st["lat"], st["p"]
    faces_i = rng.integers(0, grid.nx, m)
    faces_j = rng.integers(1, grid.ny - 1, m)
    faces_k = rng.integers(1, grid.nz - 1, m)
    d = rel[rng.integers(0, rel.size, 3 * m)]
    lon[:m] = np.mod(grid.lon0 + faces_i * grid.dlon + d[:m] * grid.dlon, 360.0)
    lat[m:2 * m] = grid.lat0 + faces_j * grid.dlat + d[m:2 * m] * grid.dlat
    p[2 * m:] = grid.plev[faces_k] * (1.0 + d[2 * m:])
    ulps = rng.integers(-3, 4, m)
    for q in range(0, m, 3):   # a few ulps off the face itself
        x = grid.lon0 + faces_i[q] * grid.dlon
        for _ in range(abs(int(ulps[q]))):
            x = np.nextafter(x, np.inf if ulps[q] > 0 else -np.inf)
        lon[q] = x
    parts = M.Particles.from_numpy(st)
    keys = ctx.cell_keys(parts).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(keys, osort.cell_keys(grid, lon, lat, p))
    ctx.sort(parts)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    ref = osort.sort_state(grid, st)
    for k in ("lon", "lat", "p", "id"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


@pytest.mark.parametrize("n", [0, 3000])
def test_all_keys_equal_keeps_the_order(M, n):
    """Every particle in one cell (one key): the stable sort leaves the arrays as they are;
    an empty set is a no-op."""
    grid = grid_2deg_20lev()
    ctx = _ctx(M, grid)
    st = uniform_particles(n, grid.plev, seed=5)
    st["lon"][:], st["lat"][:], st["p"][:] = 123.4, -56.7, 45000.0
    st["id"] = np.random.default_rng(1).permutation(n).astype(np.uint32)
    st["up"] = np.arange(n, dtype=np.float32)
    parts = M.Particles.from_numpy(st)
    ctx.sort(parts)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    for k in ("lon", "lat", "p", "id", "release", "up"):
        np.testing.assert_array_equal(got[k], st[k], err_msg=k)
