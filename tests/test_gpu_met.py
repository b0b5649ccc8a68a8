"""load_met parity: device records and scales are bit-identical to the oracle's packing."""
import numpy as np
import pytest
import torch

from oracle import met as omet
from workloads import cfg1_snapshot, fourier_modes, fourier_snapshot, grid_2deg_20lev, grid_global

from _gpu_common import M, make_ctx  # noqa: F401

pytestmark = pytest.mark.gpu


def _fields(grid, seed, with_T):
    rng = np.random.default_rng(seed)
    shp = (grid.nz, grid.ny, grid.nx)
    scale = np.logspace(-3, 2, grid.nz)[:, None, None]
    f = {k: (rng.standard_normal(shp) * scale).astype(np.float32) for k in ("u", "v", "w")}
    f["w"][3] = 0.0                    # an all-zero level -> scale 1
    if with_T:
        f["T"] = (250 + 20 * rng.standard_normal(shp)).astype(np.float32)
    return f


@pytest.mark.parametrize("storage", [omet.FP32, omet.BF16, omet.FP16])
@pytest.mark.parametrize("nvars", [3, 4])
def test_pack_bit_exact(M, storage, nvars):
    grid = grid_global(40, 33, 37)          # ragged against the 32 x 32 transpose tiles
    f = _fields(grid, 5 + storage, nvars == 4)
    ctx = make_ctx(M, grid, [f, f], [0.0, 3600.0], storage=storage, nvars=nvars)
    rec, sc, t = ctx.slot_arrays(0)
    erec, esc = omet.pack(f, storage)
    assert t == 0.0
    np.testing.assert_array_equal(sc, esc)
    np.testing.assert_array_equal(rec.view(np.uint32 if storage == omet.FP32 else np.uint16),
                                  erec.view(np.uint32 if storage == omet.FP32 else np.uint16))


@pytest.mark.parametrize("storage", [omet.FP32, omet.BF16])
def test_host_source_path_identical(M, storage):
    grid = grid_2deg_20lev()
    f = cfg1_snapshot(grid)
    a = make_ctx(M, grid, [f, f], [0.0, 1.0], storage=storage, device=True)
    b = make_ctx(M, grid, [f, f], [0.0, 1.0], storage=storage, device=False)
    ra, sa, _ = a.slot_arrays(1)
    rb, sb, _ = b.slot_arrays(1)
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(sa, sb)


def test_fourier_1deg_snapshot_packs(M):
    grid = grid_global(360, 181, 60)
    modes = fourier_modes(2)
    f = fourier_snapshot(grid, modes, 0.0, device="cuda")
    ctx = make_ctx(M, grid, [f, f], [0.0, 21600.0], storage=omet.BF16)
    rec, sc, _ = ctx.slot_arrays(0)
    erec, esc = omet.pack(f, omet.BF16)
    np.testing.assert_array_equal(sc, esc)
    np.testing.assert_array_equal(rec, erec)


def test_load_met_errors(M):
    grid = grid_2deg_20lev()
    ctx = M.Context(grid)
    u = torch.zeros(grid.nz, grid.ny, grid.nx, device="cuda")
    for bad in (3, -1):   # three slots: 0, 1, 2
        with pytest.raises(M.MptracError) as e:
            ctx.load_met(bad, 0.0, u, u, u)
        assert e.value.code == -1
    # stepping before two slots are loaded
    ctx.load_met(0, 0.0, u, u, u)
    parts = M.Particles.from_numpy({"lon": np.zeros(4), "lat": np.zeros(4), "p": np.full(4, 5e4),
                                    "id": np.arange(4, dtype=np.uint32)})
    with pytest.raises(M.MptracError) as e:
        ctx.advect(parts, 0.0, 180.0, 1)
    assert e.value.code == -7


def test_copy_probe_copies_and_checks_its_arguments(M):
    """The bandwidth probe copies its source exactly (any repetition count, a ragged element count)
    and rejects sizes that are not whole 16-byte elements and unaligned pointers on the host."""
    src = torch.arange(4 * 1_000_003, dtype=torch.float32, device="cuda")
    dst = torch.zeros_like(src)
    for reps in (1, 3):
        dst.zero_()
        M.copy_probe(src, dst, reps)
        torch.cuda.synchronize()
        assert torch.equal(dst, src)
    with pytest.raises(M.MptracError) as e:
        M.copy_probe(src[1:], dst[1:], 1)          # 4-byte offset: not 16-byte aligned
    assert e.value.code == -1
    with pytest.raises(M.MptracError):
        M.copy_probe(src[:6], dst[:6], 1)          # 24 bytes: not whole 16-byte elements
    with pytest.raises(M.MptracError):
        M.copy_probe(src, dst, 0)
