"""The fused step-and-sort hand-off is exactly mptrac_step followed by mptrac_sort.

``mptrac_step_sort`` (= ``mptrac_step_handoff`` + ``mptrac_sort_handoff``)
has the step's last launch write the final state, cell keys and first-digit
histograms into the sort workspace.  Every array must come out bit-identical
to a plain step followed by a plain sort: with and without mesoscale
diffusion, with both diffusion terms off (the advection kernel), over more
launches than one (only the last hands off), with release windows that leave
particles untouched, without the optional arrays, and at ragged sizes.
"""
import numpy as np
import pytest
import torch

from workloads import fourier_modes, fourier_snapshot, grid_2deg_20lev, uniform_particles

from _gpu_common import M, make_ctx  # noqa: F401

pytestmark = pytest.mark.gpu

T6H = 21600.0


@pytest.fixture(scope="module")
def fields():
    grid = grid_2deg_20lev()
    modes = fourier_modes(6)
    return grid, fourier_snapshot(grid, modes, 0.0), fourier_snapshot(grid, modes, T6H)


def _pair(M, ctx, st, meso, release, prm, nsteps, t0=0.0, dt=120.0):
    a = M.Particles.from_numpy(st, meso=meso, release=release)
    b = a.clone()
    ctx.step(a, t0, dt, prm, 31, 5, nsteps)
    ctx.sort(a)
    ws = torch.full((ctx.sort_workspace_bytes(b.n),), 7, dtype=torch.uint8, device="cuda")   # garbage
    ctx.step_sort(b, t0, dt, prm, 31, 5, nsteps, ws)
    torch.cuda.synchronize()
    return a.to_numpy(), b.to_numpy()


@pytest.mark.parametrize("n, meso, release, nsteps, diffusion", [
    (50_000, True, True, 20, True),
    (50_000, False, False, 20, True),
    (30_001, True, True, 20, False),
    (3_333, True, True, 130, True),
    (17, True, False, 7, True),
    (1, True, True, 3, True),
])
def test_step_sort_equals_step_then_sort(M, fields, n, meso, release, nsteps, diffusion):
    grid, f0, f1 = fields
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    st = uniform_particles(n, grid.plev, seed=n + nsteps)
    prm = M.DiffParams(turb=diffusion, meso=diffusion and meso)
    ref, got = _pair(M, ctx, st, meso, release, prm, nsteps)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    ctx.close()


def test_step_sort_with_release_windows(M, fields):
    """Particles of releases not active during the steps keep their state and are still sorted."""
    grid, f0, f1 = fields
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    n = 20_000
    st = uniform_particles(n, grid.plev, seed=77)
    rng = np.random.default_rng(77)
    st["release"] = rng.integers(0, 5, n).astype(np.uint32)
    # steps cover [0, 3600): release 0 always active, 1 starts mid-way, 2 ends mid-way, 3 never active,
    # 4 outside the table
    ctx.set_releases(np.array([0.0, 1800.0, 0.0, 5000.0]), np.array([T6H, T6H, 1800.0, T6H]))
    prm = M.DiffParams()
    ref, got = _pair(M, ctx, st, True, True, prm, 20, dt=180.0)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    untouched = np.isin(ref["release"], [3, 4])
    orig = {k: v[np.argsort(st["id"])] for k, v in st.items() if k in ("lon", "lat", "p")}
    by = np.argsort(ref["id"])
    for k in ("lon", "lat", "p"):
        np.testing.assert_array_equal(ref[k][by][untouched[by]], np.asarray(orig[k])[untouched[by]])
    ctx.close()


def test_step_sort_zero_steps_is_a_sort(M, fields):
    grid, f0, f1 = fields
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    st = uniform_particles(5000, grid.plev, seed=3)
    a = M.Particles.from_numpy(st)
    b = a.clone()
    ctx.sort(a)
    ctx.step_sort(b, 0.0, 180.0, M.DiffParams(), 1, 0, 0)
    torch.cuda.synchronize()
    ga, gb = a.to_numpy(), b.to_numpy()
    for k in ga:
        np.testing.assert_array_equal(gb[k], ga[k], err_msg=k)
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(M.MptracError) as e:
        ctx.step_sort(b, 0.0, 180.0, M.DiffParams(), 1, 0, 5, small)
    assert e.value.code == -5
    with pytest.raises(M.MptracError) as e:
        ctx.step_handoff(b, 0.0, 180.0, M.DiffParams(), 1, 0, 0, torch.empty(ctx.sort_workspace_bytes(b.n),
                                                                              dtype=torch.uint8, device="cuda"))
    assert e.value.code == -1
    ctx.close()
