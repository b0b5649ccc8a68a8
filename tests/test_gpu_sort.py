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
