"""Met sampling along trajectories (module_meteo) and particle counts per met cell (write_grid)."""
import numpy as np
import pytest
import torch

from oracle import met as omet
from oracle import meteo
from oracle import sort as osort
from workloads import fourier_modes, fourier_snapshot, grid_global, uniform_particles

from _gpu_common import M, make_ctx  # noqa: F401

pytestmark = pytest.mark.gpu
T6H = 21600.0


@pytest.mark.parametrize("storage", [omet.FP32, omet.BF16, omet.FP16])
def test_sample_met_matches_oracle(M, storage):
    grid = grid_global(90, 46, 25)
    m = fourier_modes(6, with_T=True)
    f0 = fourier_snapshot(grid, m, 0.0)
    f1 = fourier_snapshot(grid, m, T6H)
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H], storage=storage, nvars=4)
    st = uniform_particles(30_001, grid.plev, seed=9)
    parts = M.Particles.from_numpy(st, meso=False)
    t = 9000.0
    out = ctx.sample_met(parts, t).cpu().numpy()
    ref = meteo.sample(grid, omet.stored_fields(f0, storage), 0.0, omet.stored_fields(f1, storage), T6H, t,
                       st["lon"], st["lat"], st["p"])
    for i, (v, scale) in enumerate((("u", 20.0), ("v", 20.0), ("w", 0.5), ("T", 300.0))):
        err = np.abs(out[i] - ref[v]).max()
        assert err < 2e-5 * scale * 4, (v, err)


def test_sample_met_without_T_is_zero(M):
    grid = grid_global(36, 19, 10)
    f = {k: np.ones((10, 19, 36), np.float32) for k in ("u", "v", "w")}
    ctx = make_ctx(M, grid, [f, f], [0.0, 1.0])
    parts = M.Particles.from_numpy(uniform_particles(100, grid.plev, seed=1), meso=False)
    out = ctx.sample_met(parts, 0.5).cpu().numpy()
    np.testing.assert_allclose(out[:3], 1.0, rtol=1e-6)
    assert np.all(out[3] == 0)


@pytest.mark.parametrize("sort_first", [False, True])
def test_grid_counts_bit_exact(M, sort_first):
    grid = grid_global(360, 181, 60, 1e5, 1e3)
    z = {k: np.zeros((60, 181, 360), np.float32) for k in ("u", "v", "w")}
    ctx = make_ctx(M, grid, [z, z], [0.0, 1.0])
    st = uniform_particles(200_003, grid.plev, seed=10)
    st["lon"][::4], st["lat"][::4], st["p"][::4] = 100.0, 20.0, grid.plev[10]   # one crowded cell
    st["lon"][1::9] = 359.99999999999994
    parts = M.Particles.from_numpy(st, meso=False)
    if sort_first:
        ctx.sort(parts)
    counts = ctx.grid_counts(parts).cpu().numpy().view(np.uint32)
    ref = meteo.grid_counts(grid, st["lon"], st["lat"], st["p"])
    np.testing.assert_array_equal(counts, ref)
    assert counts.sum() == 200_003


@pytest.mark.parametrize("storage", [omet.FP32, omet.BF16])
def test_sedimentation_matches_oracle(M, storage):
    from oracle import sedi
    grid = grid_global(90, 46, 25)
    m = fourier_modes(7, with_T=True)
    f0 = fourier_snapshot(grid, m, 0.0)
    f1 = fourier_snapshot(grid, m, T6H)
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H], storage=storage, nvars=4)
    st = uniform_particles(20_000, grid.plev, seed=11)
    rng = np.random.default_rng(2)
    r = np.exp(rng.uniform(np.log(1e-7), np.log(2e-5), st["lon"].size)).astype(np.float32)
    rho_p = rng.uniform(800, 3000, st["lon"].size).astype(np.float32)
    parts = M.Particles.from_numpy(st, meso=False)
    ctx.sediment(parts, torch.from_numpy(r).cuda(), torch.from_numpy(rho_p).cuda(), 600.0, 60.0, 30)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    T0 = omet.stored_fields(f0, storage)["T"]
    T1 = omet.stored_fields(f1, storage)["T"]
    ref = sedi.sediment(grid, T0, 0.0, T1, T6H, st, r.astype(np.float64), rho_p.astype(np.float64), 600.0, 60.0, 30)
    dp_ref = ref - st["p"]
    dp_got = got["p"] - st["p"]
    assert np.all(dp_ref >= 0)
    # float32 physics: the pressure increments agree to 1e-4 of themselves (or 1e-3 Pa)
    np.testing.assert_allclose(dp_got, dp_ref, rtol=1e-4, atol=1e-3)
    np.testing.assert_array_equal(got["lon"], st["lon"])


def test_sedimentation_needs_temperature(M):
    grid = grid_global(36, 19, 10)
    f = {k: np.ones((10, 19, 36), np.float32) for k in ("u", "v", "w")}
    ctx = make_ctx(M, grid, [f, f], [0.0, 1.0])
    parts = M.Particles.from_numpy(uniform_particles(10, grid.plev, seed=1), meso=False)
    one = torch.ones(10, device="cuda")
    with pytest.raises(M.MptracError) as e:
        ctx.sediment(parts, one, one, 0.0, 0.1, 1)
    assert e.value.code == -1


def test_sampling_and_settling_at_degenerate_positions(M):
    """Met sampling and sedimentation from the poles, the longitude seam, grid nodes, the top
    and bottom levels and pressures outside the level range (clamped), against the oracle."""
    from oracle import sedi
    grid = grid_global(90, 46, 25)
    m = fourier_modes(8, with_T=True)
    f0, f1 = fourier_snapshot(grid, m, 0.0), fourier_snapshot(grid, m, T6H)
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H], nvars=4)
    lats = [90.0, -90.0, 89.99999, 0.0, 44.0]
    lons = [0.0, 359.99999999999994, 180.0, 4.0]
    ps = [grid.plev[0], grid.plev[-1], grid.plev[0] * 1.1, grid.plev[-1] * 0.8, grid.plev[12]]
    L = np.array([(lo, la, p) for la in lats for lo in lons for p in ps])
    st = uniform_particles(len(L), grid.plev, seed=3)
    st["lon"], st["lat"], st["p"] = L[:, 0].copy(), L[:, 1].copy(), L[:, 2].copy()
    parts = M.Particles.from_numpy(st, meso=False)
    out = ctx.sample_met(parts, 5400.0).cpu().numpy()
    ref = meteo.sample(grid, f0, 0.0, f1, T6H, 5400.0, st["lon"], st["lat"], st["p"])
    for i, (v, scale) in enumerate((("u", 20.0), ("v", 20.0), ("w", 0.5), ("T", 300.0))):
        assert np.all(np.isfinite(out[i])), v
        assert np.abs(out[i] - ref[v]).max() < 8e-5 * scale, v
    r = np.full(len(L), 5e-6, np.float32)
    rho_p = np.full(len(L), 2000.0, np.float32)
    ctx.sediment(parts, torch.from_numpy(r).cuda(), torch.from_numpy(rho_p).cuda(), 600.0, 60.0, 10)
    torch.cuda.synchronize()
    got = parts.to_numpy()
    refp = sedi.sediment(grid, f0["T"], 0.0, f1["T"], T6H, st, r.astype(np.float64), rho_p.astype(np.float64),
                         600.0, 60.0, 10)
    assert np.all(np.isfinite(got["p"]))
    np.testing.assert_allclose(got["p"], refp, rtol=1e-4)
    assert np.all((got["p"] >= grid.plev[-1]) & (got["p"] <= grid.plev[0]))


@pytest.mark.parametrize("storage", [omet.FP32, omet.BF16])
def test_masked_advection_matches_oracle(M, storage):
    """mptrac_advect_masked (the surrogate's plain fallback): the particles whose mask is set take
    the plain midpoint steps of the oracle, and the others are left exactly as they were.  The mask
    is random, then a block of whole warps, then empty and full."""
    from _gpu_common import assert_positions_close
    from oracle import transport as tr
    grid = grid_global(90, 46, 25)
    m = fourier_modes(7)
    f0, f1 = fourier_snapshot(grid, m, 0.0), fourier_snapshot(grid, m, T6H)
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H], storage=storage)
    met = tr.Met(grid, 0.0, omet.stored_fields(f0, storage), T6H, omet.stored_fields(f1, storage))
    n = 20_003
    st = uniform_particles(n, grid.plev, seed=13)
    rng = np.random.default_rng(14)
    masks = [rng.random(n) < 0.14, (np.arange(n) // 32) % 5 == 0, np.zeros(n, bool), np.ones(n, bool)]
    for mask in masks:
        parts = M.Particles.from_numpy(st, meso=False, release=False)
        M.advect_masked(ctx, parts, torch.from_numpy(mask.astype(np.uint8)).cuda(), 3600.0, 180.0, 10)
        torch.cuda.synchronize()
        got = parts.to_numpy()
        for k in ("lon", "lat", "p"):
            np.testing.assert_array_equal(got[k][~mask], st[k][~mask], err_msg=k)
        if mask.any():
            sub = {k: v[mask] for k, v in st.items()}
            ref = tr.advect(met, sub, 3600.0, 180.0, 10)
            assert_positions_close({k: v[mask] for k, v in got.items()}, ref, what=f"masked advection, storage {storage}")


def test_colstats_match_numpy(M):
    """Column means and standard deviations of a float32 device matrix against numpy in float64,
    with the floor that turns the standard deviation of a constant column into 1."""
    rng = np.random.default_rng(15)
    n, ncol = 300_001, 176
    X = (rng.standard_normal((n, ncol)) * rng.uniform(0.01, 100, ncol) + rng.uniform(-50, 50, ncol)).astype(np.float32)
    X[:, 170:] = 0.0
    X[:, 100] = 3.25                       # constant, non-zero
    mean, sd = M.colstats(torch.from_numpy(X).cuda())
    ref_m = X.astype(np.float64).mean(axis=0)
    ref_s = X.astype(np.float64).std(axis=0)
    np.testing.assert_allclose(mean, ref_m, rtol=1e-6, atol=1e-6 * np.abs(X).max())
    varying = ref_s > 0
    np.testing.assert_allclose(sd[varying], ref_s[varying], rtol=1e-5)
    assert np.all(sd[~varying] == 1.0) and not varying[100] and np.all(~varying[170:])
    with pytest.raises(M.MptracError):
        M.colstats(torch.zeros((0, 4), dtype=torch.float32, device="cuda"))


def test_every_particle_call_accepts_zero_particles(M):
    """n = 0 through every entry point that takes particles: nothing is launched on the
    particle arrays and nothing faults; fixed-size outputs are still written (grid counts zero)."""
    grid = grid_global(36, 19, 8)
    z = {k: np.full((grid.nz, grid.ny, grid.nx), 250.0 if k == "T" else 1.0, np.float32) for k in ("u", "v", "w", "T")}
    ctx = make_ctx(M, grid, [z, z], [0.0, T6H], nvars=4)
    empty = {"lon": np.zeros(0), "lat": np.zeros(0), "p": np.zeros(0), "id": np.zeros(0, np.uint32)}
    parts = M.Particles.from_numpy(empty)
    ctx.advect(parts, 0.0, 180.0, 3)
    ctx.step(parts, 0.0, 180.0, M.DiffParams(), 1, 0, 3)
    ctx.sort(parts)
    assert ctx.sample_met(parts, 0.0).numel() == 0
    counts = ctx.grid_counts(parts)
    assert counts.numel() == grid.nx * grid.ny * grid.nz and int(counts.sum().item()) == 0
    zf = torch.zeros(0, dtype=torch.float32, device="cuda")
    ctx.sediment(parts, zf, zf, 0.0, 60.0, 2)
    assert ctx.cell_keys(parts).numel() == 0
    M.advect_masked(ctx, parts, torch.zeros(0, dtype=torch.uint8, device="cuda"), 0.0, 180.0, 2)
    assert M.surr_features(ctx, parts, 0.0).shape[0] == 0
    sur = M.Surrogate(64)
    sur.advance(ctx, parts, 0.0, 1800.0, torch.zeros(0, dtype=torch.uint8, device="cuda"))
    sur.status()
    torch.cuda.synchronize()
    assert parts.n == 0
