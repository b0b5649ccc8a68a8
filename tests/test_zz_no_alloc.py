"""The allocation-free sort entry point gives exactly the result of the ordinary one.

mptrac_sort_noalloc exists for callers that may not allocate device memory --
for example a host whose device heap belongs to another framework's pool
allocator, or a pipeline in which the implicit device synchronisation of
cudaMalloc is not allowed.  It sorts with a fixed static scratch array inside
the library instead of a caller workspace.  This file is named so that pytest
collects it last; it also passes when run on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

from workloads import grid_1deg_60lev, uniform_particles

from _gpu_common import M, make_ctx  # noqa: F401

pytestmark = pytest.mark.gpu


def _noalloc(M, ctx, parts):
    lib = M.load()
    rc = lib.mptrac_sort_noalloc(ctx.h, ctypes.byref(parts.desc()), torch.cuda.current_stream().cuda_stream)
    return rc


def test_noalloc_sort_matches_workspace_sort_twice(M):
    grid = grid_1deg_60lev()
    z = {k: np.zeros((grid.nz, grid.ny, grid.nx), np.float32) for k in ("u", "v", "w")}
    ctx = make_ctx(M, grid, [z, z], [0.0, 1.0])
    nmax = 262144
    for call, (n, seed) in enumerate(((200_003, 21), (nmax, 22))):
        st = uniform_particles(n, grid.plev, seed=seed)
        st["lon"][::9] = 120.0          # repeated keys exercise stability
        st["up"] = np.arange(n, dtype=np.float32)
        a = M.Particles.from_numpy(st)
        b = M.Particles.from_numpy(st)
        assert _noalloc(M, ctx, a) == 0, M.load().mptrac_last_error(None)
        ctx.sort(b)                     # the ordinary entry point with a workspace
        torch.cuda.synchronize()
        ga, gb = a.to_numpy(), b.to_numpy()
        for k in ("lon", "lat", "p", "id", "release", "up", "vp", "wp"):
            np.testing.assert_array_equal(ga[k], gb[k], err_msg=f"call {call}: {k}")
        assert not np.array_equal(ga["id"], st["id"])   # it really sorted


def test_noalloc_sort_rejects_oversize(M):
    grid = grid_1deg_60lev()
    z = {k: np.zeros((grid.nz, grid.ny, grid.nx), np.float32) for k in ("u", "v", "w")}
    ctx = make_ctx(M, grid, [z, z], [0.0, 1.0])
    st = uniform_particles(262145, grid.plev, seed=3)
    a = M.Particles.from_numpy(st)
    assert _noalloc(M, ctx, a) == -1
    assert b"at most" in M.load().mptrac_last_error(None)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.to_numpy()["id"], st["id"])   # untouched
