"""Trajectory parity of the advect / diffuse / step kernels against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import met as omet
from oracle import sort as osort
from oracle import transport as tr
from workloads import (cfg1_snapshot, column_releases, fourier_modes, fourier_snapshot,
                       grid_2deg_20lev, grid_global, uniform_particles)

from _gpu_common import M, TOL_DEG, TOL_P, assert_positions_close, by_id, make_ctx  # noqa: F401

pytestmark = pytest.mark.gpu
T6H = 21600.0


@pytest.fixture(scope="module")
def cfg1(M):
    grid = grid_2deg_20lev()
    snap = cfg1_snapshot(grid)
    ctx = make_ctx(M, grid, [snap, snap], [0.0, T6H])
    met = tr.Met(grid, 0.0, snap, T6H, snap)
    return grid, ctx, met


def test_cfg1_advect_120_steps_within_tolerance(M, cfg1):
    """2 degree analytic case, 1e4 particles, dt = 180 s, 120 steps."""
    grid, ctx, met = cfg1
    st0 = uniform_particles(10_000, grid.plev, seed=1)
    parts = M.Particles.from_numpy(st0)
    ctx.advect(parts, 0.0, 180.0, 120)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    ref = tr.advect(met, st0, 0.0, 180.0, 120)
    assert_positions_close(got, ref, what="cfg1 advect")
    np.testing.assert_array_equal(got["id"], st0["id"])


def test_chunked_launches_equal_single(M):
    """200 steps (two kernel launches internally) and 3 x ~67 steps agree with the oracle."""
    grid = grid_2deg_20lev()
    snap = cfg1_snapshot(grid)
    ctx = make_ctx(M, grid, [snap, snap], [0.0, 2 * T6H])
    met = tr.Met(grid, 0.0, snap, 2 * T6H, snap)
    st0 = uniform_particles(3001, grid.plev, seed=11)
    a = M.Particles.from_numpy(st0)
    b = M.Particles.from_numpy(st0)
    ctx.advect(a, 0.0, 180.0, 200)
    for t0, n in ((0.0, 67), (67 * 180.0, 67), (134 * 180.0, 66)):
        ctx.advect(b, t0, 180.0, n)
    torch.cuda.synchronize()
    ref = tr.advect(met, st0, 0.0, 180.0, 200)
    assert_positions_close(a.to_numpy(), ref, what="200 steps single")
    assert_positions_close(b.to_numpy(), ref, what="200 steps chunked")


@pytest.fixture(scope="module")
def fourier(M):
    grid = grid_global(120, 61, 30)
    m = fourier_modes(2)
    f0 = fourier_snapshot(grid, m, 0.0)
    f1 = fourier_snapshot(grid, m, T6H)
    return grid, f0, f1


@pytest.mark.parametrize("storage", [omet.FP32, omet.BF16, omet.FP16])
@pytest.mark.parametrize("mode", ["advect", "diffuse", "step"])
def test_fourier_modes_parity(M, fourier, storage, mode):
    grid, f0, f1 = fourier
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H], storage=storage)
    met = tr.Met(grid, 0.0, omet.stored_fields(f0, storage), T6H, omet.stored_fields(f1, storage))
    st0 = uniform_particles(20_000, grid.plev, seed=3)
    parts = M.Particles.from_numpy(st0)
    prm = M.DiffParams()
    t, dt, ns = 3600.0, 180.0, 20
    if mode == "advect":
        ctx.advect(parts, t, dt, ns)
        ref = tr.advect(met, st0, t, dt, ns)
    elif mode == "diffuse":
        ctx.diffuse(parts, t, dt, prm, 99, 40, ns)
        ref = tr.diffuse(met, st0, t, dt, tr.DiffParams(), 99, 40, ns)
    else:
        ctx.step(parts, t, dt, prm, 99, 40, ns)
        ref = tr.step(met, st0, t, dt, tr.DiffParams(), 99, 40, ns)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    assert_positions_close(got, ref, what=f"{mode} storage {storage}",
                           lon_metric="deg" if mode == "advect" else "arc")
    if mode != "advect":
        for k in ("up", "vp", "wp"):
            scale = np.abs(ref[k]).max() + 1e-30
            assert np.abs(got[k] - ref[k]).max() <= 1e-4 * scale, k


def test_release_windows(M, fourier):
    grid, f0, f1 = fourier
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    met = tr.Met(grid, 0.0, f0, T6H, f1)
    rel = column_releases(16, seed=4, count_scale=2e-3)
    st0 = rel.particles
    ts = np.linspace(0, 3000, 16)
    te = ts + np.linspace(500, 4000, 16)
    ts[3], te[3] = 1e9, 2e9             # never active
    ctx.set_releases(ts, te)
    parts = M.Particles.from_numpy(st0)
    prm = M.DiffParams()
    ctx.step(parts, 0.0, 180.0, prm, 5, 0, 30)
    torch.cuda.synchronize()
    ref = tr.step(met, st0, 0.0, 180.0, tr.DiffParams(), 5, 0, 30, windows=(ts, te))
    got = parts.to_numpy()
    assert_positions_close(got, ref, what="release windows", lon_metric="arc")
    still = st0["release"] == 3
    np.testing.assert_array_equal(got["lon"][still], st0["lon"][still])
    ctx.set_releases([], [])


def test_fused_identities(M, fourier):
    grid, f0, f1 = fourier
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    st0 = uniform_particles(5000, grid.plev, seed=8)
    a, b = M.Particles.from_numpy(st0), M.Particles.from_numpy(st0)
    off = M.DiffParams(turb=False, meso=False)
    ctx.advect(a, 0.0, 180.0, 15)
    ctx.step(b, 0.0, 180.0, off, 1, 0, 15)
    torch.cuda.synchronize()
    for k in ("lon", "lat", "p"):
        np.testing.assert_array_equal(getattr(a, k).cpu().numpy(), getattr(b, k).cpu().numpy())
    zero = {k: np.zeros_like(v) for k, v in f0.items()}
    ctx0 = make_ctx(M, grid, [zero, zero], [0.0, T6H])
    c, d = M.Particles.from_numpy(st0), M.Particles.from_numpy(st0)
    prm = M.DiffParams(meso=False)
    ctx0.diffuse(c, 0.0, 180.0, prm, 3, 0, 15)
    ctx0.step(d, 0.0, 180.0, prm, 3, 0, 15)
    torch.cuda.synchronize()
    for k in ("lon", "lat", "p"):
        np.testing.assert_allclose(getattr(c, k).cpu().numpy(), getattr(d, k).cpu().numpy(), rtol=1e-12, atol=1e-9)


def test_sort_invariance_bit_exact(M, fourier):
    """step(sort(P)) == sort(step(P)) exactly: results depend on particle id, not slot."""
    grid, f0, f1 = fourier
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    st0 = uniform_particles(30_000, grid.plev, seed=9)
    a, b = M.Particles.from_numpy(st0), M.Particles.from_numpy(st0)
    prm = M.DiffParams()
    ctx.sort(a)
    ctx.step(a, 0.0, 180.0, prm, 17, 0, 20)
    ctx.step(b, 0.0, 180.0, prm, 17, 0, 20)
    ctx.sort(b)
    torch.cuda.synchronize()
    ga, gb = by_id(a.to_numpy()), by_id(b.to_numpy())
    for k in ("lon", "lat", "p", "up", "vp", "wp"):
        np.testing.assert_array_equal(ga[k], gb[k])


@pytest.mark.parametrize("n", [0, 1, 255, 257])
def test_small_and_ragged_counts(M, cfg1, n):
    grid, ctx, met = cfg1
    st0 = uniform_particles(n, grid.plev, seed=12)
    parts = M.Particles.from_numpy(st0)
    ctx.step(parts, 0.0, 180.0, M.DiffParams(), 1, 0, 12)
    torch.cuda.synchronize()
    if n:
        ref = tr.step(met, st0, 0.0, 180.0, tr.DiffParams(), 1, 0, 12)
        assert_positions_close(parts.to_numpy(), ref, what=f"n={n}", lon_metric="arc")


def test_host_validation_errors(M, cfg1):
    grid, ctx, met = cfg1
    st0 = uniform_particles(10, grid.plev, seed=2)
    parts = M.Particles.from_numpy(st0)
    with pytest.raises(M.MptracError) as e:
        ctx.advect(parts, 0.0, 180.0, 121)       # leaves [0, 6 h]
    assert e.value.code == -4
    with pytest.raises(M.MptracError) as e:
        ctx.advect(parts, 0.0, -1.0, 1)
    assert e.value.code == -1
    noms = M.Particles.from_numpy(st0, meso=False)
    with pytest.raises(M.MptracError) as e:
        ctx.step(noms, 0.0, 180.0, M.DiffParams(), 1, 0, 1)
    assert e.value.code == -1
    host = M.Particles(*(torch.from_numpy(np.ascontiguousarray(v)) for v in
                         (st0["lon"], st0["lat"], st0["p"], st0["id"].view(np.int32))))
    with pytest.raises(M.MptracError) as e:
        ctx.advect(host, 0.0, 180.0, 1)
    assert e.value.code == -1
    ctx.advect(parts, 0.0, 180.0, 0)             # no steps: no-op
    torch.cuda.synchronize()
    np.testing.assert_array_equal(parts.lon.cpu().numpy(), st0["lon"])
    from paper_2211_12616_gb300 import _native
    for variant, schedule in ((7, 0), (-1, 0), (2, 65), (2, -1)):
        with pytest.raises(M.MptracError) as e:
            _native.check(M.load().mptrac_set_launch(ctx.h, variant, schedule), ctx.h)
        assert e.value.code == -1
    with pytest.raises(ValueError):
        ctx.set_launch(2, True, per_thread=2)
    # particle counts outside [0, 2^31 - 1] are rejected before any launch
    import ctypes
    lib = M.load()
    for bad_n in (-1, 2 ** 31):
        d = parts.desc()
        d.n = bad_n
        assert lib.mptrac_advect(ctx.h, ctypes.byref(d), 0.0, 180.0, 1, torch.cuda.current_stream().cuda_stream) == -1
        assert lib.mptrac_step(ctx.h, ctypes.byref(d), 0.0, 180.0, ctypes.byref(M.DiffParams().desc()), 1, 0, 1,
                               torch.cuda.current_stream().cuda_stream) == -1
        assert b"out of range" in lib.mptrac_last_error(ctx.h)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(parts.lon.cpu().numpy(), st0["lon"])


def test_checkpoint_resume_bit_identical(M, fourier):
    """Stopping after 20 steps, copying the state to the host and back, and resuming with the
    global step index gives exactly the uninterrupted run (counter-based random numbers)."""
    grid, f0, f1 = fourier
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    st0 = uniform_particles(10_000, grid.plev, seed=21)
    prm = M.DiffParams()
    a = M.Particles.from_numpy(st0)
    ctx.step(a, 0.0, 180.0, prm, 77, 0, 40)
    b = M.Particles.from_numpy(st0)
    ctx.step(b, 0.0, 180.0, prm, 77, 0, 20)
    torch.cuda.synchronize()
    saved = b.to_numpy()                       # checkpoint: the whole particle state on the host
    c = M.Particles.from_numpy(saved)          # restart in fresh device arrays
    ctx.step(c, 20 * 180.0, 180.0, prm, 77, 20, 20)
    torch.cuda.synchronize()
    ga, gc = a.to_numpy(), c.to_numpy()
    for k in ("lon", "lat", "p", "up", "vp", "wp", "id"):
        np.testing.assert_array_equal(ga[k], gc[k], err_msg=k)


def test_fused_step_over_launch_limit(M, fourier):
    """300 fused steps in one call run as launches of 128, 128 and 44 steps (the time-weight
    table of one launch holds 128); the result matches the oracle and three calls of 100."""
    grid, f0, f1 = fourier
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    met = tr.Met(grid, 0.0, f0, T6H, f1)
    st0 = uniform_particles(3001, grid.plev, seed=31)
    prm = M.DiffParams()
    a, b = M.Particles.from_numpy(st0), M.Particles.from_numpy(st0)
    ctx.step(a, 0.0, 60.0, prm, 17, 0, 300)
    for k in range(3):
        ctx.step(b, k * 6000.0, 60.0, prm, 17, 100 * k, 100)
    torch.cuda.synchronize()
    ga, gb = a.to_numpy(), b.to_numpy()
    for k in ("lon", "lat", "p", "up", "vp", "wp"):
        np.testing.assert_array_equal(ga[k], gb[k], err_msg=k)
    ref = tr.step(met, st0, 0.0, 60.0, tr.DiffParams(), 17, 0, 300)
    assert_positions_close(ga, ref, what="300 fused steps", lon_metric="arc")


def test_maximum_level_count(M):
    """MPTRAC_MAX_NZ = 256 levels: fused steps with diffusion and the sort keys against the
    oracle (the shared level tables and the level search at their largest)."""
    grid = grid_global(36, 19, 256, 1e5, 10.0)
    m = fourier_modes(5)
    f0, f1 = fourier_snapshot(grid, m, 0.0), fourier_snapshot(grid, m, T6H)
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    met = tr.Met(grid, 0.0, f0, T6H, f1)
    st0 = uniform_particles(2000, grid.plev, seed=33)
    parts = M.Particles.from_numpy(st0)
    ctx.step(parts, 600.0, 180.0, M.DiffParams(), 23, 0, 20)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    ref = tr.step(met, st0, 600.0, 180.0, tr.DiffParams(), 23, 0, 20)
    assert_positions_close(got, ref, what="256 levels", lon_metric="arc")
    keys = ctx.cell_keys(parts).cpu().numpy()
    np.testing.assert_array_equal(keys, osort.cell_keys(grid, got["lon"], got["lat"], got["p"]))


def test_degenerate_positions(M, fourier):
    """Fused steps with diffusion from the degenerate places of the method: exactly on and
    within metres of the poles (diffusion carries particles over the pole: reflection and
    longitude + 180), on the longitude seam, on the top and bottom levels and outside the
    level range (clamped).  Against the oracle, by great-circle distance."""
    grid, f0, f1 = fourier
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    met = tr.Met(grid, 0.0, f0, T6H, f1)
    lats = [90.0, -90.0, 89.9999, -89.9999, 89.999999, 0.0, 45.0]
    lons = [0.0, 359.99999999999994, 180.0, 3.0]
    ps = [grid.plev[0], grid.plev[-1], grid.plev[0] * 1.05, grid.plev[-1] * 0.9, 50000.0]
    L = np.array([(lo, la, p) for la in lats for lo in lons for p in ps])
    n = len(L)
    st0 = uniform_particles(n, grid.plev, seed=41)
    st0["lon"], st0["lat"], st0["p"] = L[:, 0].copy(), L[:, 1].copy(), L[:, 2].copy()
    parts = M.Particles.from_numpy(st0)
    ctx.step(parts, 0.0, 180.0, M.DiffParams(), 29, 0, 12)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    ref = tr.step(met, st0, 0.0, 180.0, tr.DiffParams(), 29, 0, 12)
    assert_positions_close(got, ref, what="degenerate positions", lon_metric="arc")
    assert np.all(np.abs(got["lat"]) <= 90.0)
    assert np.all((got["lon"] >= 0.0) & (got["lon"] < 360.0))
    assert np.all((got["p"] >= grid.plev[-1]) & (got["p"] <= grid.plev[0]))
    # some particles did cross a pole (their longitude moved by about 180 degrees)
    dlon = np.abs(((got["lon"] - st0["lon"]) + 180.0) % 360.0 - 180.0)
    near_pole = np.abs(st0["lat"]) > 89.99
    assert np.any(dlon[near_pole] > 90.0)


@pytest.mark.parametrize("dt", [180.0, 3600.0])
def test_minimum_grid_and_long_steps(M, dt):
    """The smallest grid the ABI accepts (2 x 2 x 2: two meridians, the two poles, two levels)
    with random winds, and steps of an hour: fused steps with diffusion and the sort keys
    against the oracle.  With hour-long steps the particles stay within 80 degrees of the
    equator: closer to a pole one step turns the longitude by a large part of a circle, and
    the trajectory over several steps amplifies float32 rounding beyond the tolerance (one
    step still agrees to 3e-7 degrees there)."""
    grid = grid_global(2, 2, 2, 1e5, 1e3)
    rng = np.random.default_rng(5)
    snaps = [{k: (rng.standard_normal((2, 2, 2)) * s).astype(np.float32)
              for k, s in (("u", 20.0), ("v", 10.0), ("w", 0.3))} for _ in range(2)]
    ctx = make_ctx(M, grid, snaps, [0.0, T6H])
    met = tr.Met(grid, 0.0, snaps[0], T6H, snaps[1])
    st0 = uniform_particles(3000, grid.plev, seed=7, lat_max=80.0 if dt > 1000.0 else 90.0)
    parts = M.Particles.from_numpy(st0)
    nsteps = 5 if dt > 1000.0 else 20
    ctx.step(parts, 0.0, dt, M.DiffParams(), 3, 0, nsteps)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    ref = tr.step(met, st0, 0.0, dt, tr.DiffParams(), 3, 0, nsteps)
    assert_positions_close(got, ref, what=f"2x2x2 grid, dt {dt}", lon_metric="arc")
    keys = ctx.cell_keys(parts).cpu().numpy()
    np.testing.assert_array_equal(keys, osort.cell_keys(grid, got["lon"], got["lat"], got["p"]))


def test_step_counter_wraps_at_32_bits(M, fourier):
    """The random-number counter takes the low 32 bits of step0 + n: a run whose global step
    crosses 2^32 matches the oracle, whose counter words are 32-bit too."""
    grid, f0, f1 = fourier
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    met = tr.Met(grid, 0.0, f0, T6H, f1)
    st0 = uniform_particles(2000, grid.plev, seed=43)
    parts = M.Particles.from_numpy(st0)
    step0 = 2**32 - 3
    ctx.step(parts, 0.0, 180.0, M.DiffParams(), 11, step0, 6)
    torch.cuda.synchronize()
    ref = tr.step(met, st0, 0.0, 180.0, tr.DiffParams(), 11, step0, 6)
    assert_positions_close(parts.to_numpy(), ref, what="step counter wrap", lon_metric="arc")


def test_increment_larger_than_the_coordinate(M, fourier):
    """Positions within one step's increment of lon0 and of the south pole (latitude is carried
    as lat - lat0), where the float-float add takes an increment larger than the coordinate and
    its Fast2Sum error term is no longer exact (off by at most half an ulp of the increment):
    10 fused steps against the oracle stay within 1e-5 degrees, ten times inside the transport
    tolerance, and the longitude criterion is literal away from the pole."""
    grid, f0, f1 = fourier
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    met = tr.Met(grid, 0.0, f0, T6H, f1)
    lons = [1e-12, 1e-9, 1e-6, 1e-3, 359.9999999999, 359.999]
    lats = [-90.0 + 1e-12, -90.0 + 1e-9, -90.0 + 1e-6, -89.999, -30.0, 0.0, 45.0]
    L = np.array([(lo, la) for la in lats for lo in lons])
    st0 = uniform_particles(len(L), grid.plev, seed=43)
    st0["lon"], st0["lat"] = L[:, 0].copy(), L[:, 1].copy()
    for diffuse in (False, True):
        parts = M.Particles.from_numpy(st0)
        prm = M.DiffParams(turb=diffuse, meso=diffuse)
        ctx.step(parts, 0.0, 180.0, prm, 11, 0, 10)
        torch.cuda.synchronize()
        got = parts.to_numpy()
        oprm = tr.DiffParams(turb=diffuse, meso=diffuse)
        ref = tr.step(met, st0, 0.0, 180.0, oprm, 11, 0, 10)
        assert_positions_close(got, ref, tol_deg=1e-5, what=f"increment > coordinate, diffusion {diffuse}",
                               lon_metric="arc")
        away = np.abs(st0["lat"]) < 80.0
        sub = {k: v[away] for k, v in got.items()}
        assert_positions_close(sub, {k: v[away] for k, v in ref.items()}, tol_deg=1e-5,
                               what="increment > coordinate, literal longitude")
