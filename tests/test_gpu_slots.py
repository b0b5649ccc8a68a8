"""Three met slots: a call uses the two loaded snapshots that bracket its time range.

A context holds three slots so that the next snapshot can be loaded while the
current interval is in use.  A step over [6 h, 12 h] on a context holding
0 h, 6 h and 12 h must give exactly what a context holding only 6 h and 12 h
gives (both with the earlier snapshot in the lower slot); a range that spans
two intervals is rejected, and so is a call with one snapshot loaded.
"""
import numpy as np
import pytest
import torch

from workloads import fourier_modes, fourier_snapshot, grid_2deg_20lev, uniform_particles

from _gpu_common import M  # noqa: F401

pytestmark = pytest.mark.gpu

T6H = 21600.0


def _snaps():
    grid = grid_2deg_20lev()
    modes = fourier_modes(8)
    return grid, [{k: torch.from_numpy(v).cuda() for k, v in fourier_snapshot(grid, modes, h * T6H).items()}
                  for h in range(3)]


def _ctx(M, grid, snaps, loads):
    ctx = M.Context(grid, M.MPTRAC_FP32)
    for slot, h in loads:
        f = snaps[h]
        ctx.load_met(slot, h * T6H, f["u"], f["v"], f["w"])
    return ctx


def test_three_slots_bracket_the_step_range(M):
    grid, snaps = _snaps()
    st = uniform_particles(20_000, grid.plev, seed=12)
    prm = M.DiffParams()
    ref_ctx = _ctx(M, grid, snaps, [(0, 1), (1, 2)])
    ctx3 = _ctx(M, grid, snaps, [(0, 0), (1, 1), (2, 2)])
    a = M.Particles.from_numpy(st)
    b = a.clone()
    ref_ctx.step(a, T6H, 180.0, prm, 5, 120, 120)
    ctx3.step(b, T6H, 180.0, prm, 5, 120, 120)
    torch.cuda.synchronize()
    ga, gb = a.to_numpy(), b.to_numpy()
    for k in ga:
        np.testing.assert_array_equal(gb[k], ga[k], err_msg=k)
    # the first interval of the three-slot context matches a two-slot context of 0 h and 6 h
    c = M.Particles.from_numpy(st)
    d = c.clone()
    ref0 = _ctx(M, grid, snaps, [(0, 0), (1, 1)])
    ref0.advect(c, 0.0, 180.0, 120)
    ctx3.advect(d, 0.0, 180.0, 120)
    torch.cuda.synchronize()
    for k in ("lon", "lat", "p"):
        np.testing.assert_array_equal(d.to_numpy()[k], c.to_numpy()[k], err_msg=k)
    # a range over two intervals, and times outside every interval
    with pytest.raises(M.MptracError) as e:
        ctx3.advect(d, 0.0, 180.0, 200)
    assert e.value.code == -4
    with pytest.raises(M.MptracError) as e:
        ctx3.advect(d, 3 * T6H, 180.0, 1)
    assert e.value.code == -4
    for ctx in (ref_ctx, ctx3, ref0):
        ctx.close()


def test_one_snapshot_is_not_an_interval(M):
    grid, snaps = _snaps()
    ctx = _ctx(M, grid, snaps, [(2, 1)])
    p = M.Particles.from_numpy(uniform_particles(10, grid.plev, seed=1))
    with pytest.raises(M.MptracError) as e:
        ctx.advect(p, T6H, 180.0, 1)
    assert e.value.code == -7
    with pytest.raises(M.MptracError) as e:
        ctx.load_met(3, 0.0, snaps[0]["u"], snaps[0]["v"], snaps[0]["w"])
    assert e.value.code == -1
    ctx.close()
