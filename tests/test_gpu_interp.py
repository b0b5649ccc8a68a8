"""4D interpolation parity (float32 kernels vs the float64 oracle)."""
import numpy as np
import pytest
import torch

from oracle import met as omet
from oracle import transport as tr
from workloads import fourier_modes, fourier_snapshot, grid_2deg_20lev, grid_global

from _gpu_common import M, make_ctx  # noqa: F401

pytestmark = pytest.mark.gpu


def _points(n, grid, seed):
    rng = np.random.default_rng(seed)
    lon = rng.uniform(0, 360, n)
    lat = rng.uniform(-90, 90, n)
    p = np.exp(rng.uniform(np.log(grid.plev[-1]) - 0.2, np.log(grid.plev[0]) + 0.2, n))
    lon[:4] = [0.0, 359.9999999, 180.0, 358.0]      # seam and nodes
    lat[:4] = [-90.0, 90.0, 0.0, 89.99]
    return lon, lat, p


@pytest.mark.parametrize("storage", [omet.FP32, omet.BF16, omet.FP16])
def test_interp_matches_oracle(M, storage):
    grid = grid_global(72, 37, 19)
    m = fourier_modes(3)
    f0 = fourier_snapshot(grid, m, 0.0)
    f1 = fourier_snapshot(grid, m, 21600.0)
    ctx = make_ctx(M, grid, [f0, f1], [0.0, 21600.0], storage=storage)
    met = tr.Met(grid, 0.0, omet.stored_fields(f0, storage), 21600.0, omet.stored_fields(f1, storage))
    n = 50_001
    lon, lat, p = _points(n, grid, 4)
    for t in (0.0, 7777.0, 21600.0):
        u, v, w, var = ctx.interp(*(torch.from_numpy(a).cuda() for a in (lon, lat, p)), t)
        ref = met.wind(lon, lat, p, t, sigma=True)
        for got, r, scale in ((u, ref[0], 20.0), (v, ref[1], 20.0), (w, ref[2], 0.5)):
            err = np.abs(got.cpu().numpy() - r).max()
            # float32 arithmetic on values of size ~4x the rms, locations rounded to float32
            assert err < 2e-5 * scale, err
        vv = var.cpu().numpy()
        for c, scale in zip(range(3), (20.0, 20.0, 0.5)):
            assert np.abs(vv[c] - ref[3 + c]).max() < 2e-5 * scale ** 2


def test_trilinear_field_exact_in_float32(M):
    grid = grid_2deg_20lev()
    lon = grid.lons[None, None, :]
    lat = grid.lats[None, :, None]
    pp = grid.plev[:, None, None]
    f = {"u": (3.0 + 0.01 * lon + 0.02 * lat + 1e-5 * pp) * np.ones((grid.nz, 1, 1)),
         "v": (0.5 * lat) * np.ones((grid.nz, 1, grid.nx)),
         "w": (1e-5 * pp) * np.ones((1, grid.ny, grid.nx))}
    f = {k: np.ascontiguousarray(np.broadcast_to(v, (grid.nz, grid.ny, grid.nx)), dtype=np.float32)
         for k, v in f.items()}
    ctx = make_ctx(M, grid, [f, f], [0.0, 1.0])
    rng = np.random.default_rng(1)
    n = 10000
    lo, la = rng.uniform(0, 357.9, n), rng.uniform(-90, 90, n)
    p = np.exp(rng.uniform(np.log(1e3), np.log(1e5), n))
    u, v, w, _ = ctx.interp(*(torch.from_numpy(a).cuda() for a in (lo, la, p)), 0.5)
    np.testing.assert_allclose(u.cpu().numpy(), 3.0 + 0.01 * lo + 0.02 * la + 1e-5 * p, atol=2e-5)
    np.testing.assert_allclose(v.cpu().numpy(), 0.5 * la, atol=2e-5)
    np.testing.assert_allclose(w.cpu().numpy(), 1e-5 * p, rtol=2e-6, atol=1e-6)
