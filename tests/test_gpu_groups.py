"""Particle groups on separate streams give bit-identical trajectories.

``Simulation(groups=G)`` sorts and steps G contiguous particle groups on
streams of their own.  Each particle's trajectory depends only on its own
state and id, so after two met intervals (one join before the second met
load) every particle must have exactly the state of the single-group run.
"""
import numpy as np
import pytest
import torch

from workloads import fourier_modes, fourier_snapshot, grid_2deg_20lev, uniform_particles

from _gpu_common import M  # noqa: F401

pytestmark = pytest.mark.gpu

DT, DT_MET = 180.0, 21600.0


def _run(M, grid, snaps, st0, groups):
    from paper_2211_12616_gb300.simulation import Simulation, periodic_snapshots
    ctx = M.Context(grid, M.MPTRAC_FP32)
    parts = M.Particles.from_numpy(st0)
    sim = Simulation(ctx, periodic_snapshots(snaps, DT_MET), DT_MET, parts, DT, M.DiffParams(), 9, 20,
                     groups=groups)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert sim.run(0.0, 2 * DT_MET, stream=s) == 240
    torch.cuda.synchronize()
    got = parts.to_numpy()
    ctx.close()
    order = np.argsort(got["id"])
    return {k: v[order] for k, v in got.items()}


@pytest.mark.parametrize("groups", [2, 3])
def test_groups_match_single_stream(M, groups):
    grid = grid_2deg_20lev()
    modes = fourier_modes(4)
    snaps = [fourier_snapshot(grid, modes, h * DT_MET, device="cuda", as_numpy=False) for h in range(3)]
    st0 = uniform_particles(30_001, grid.plev, 13)
    ref = _run(M, grid, snaps, st0, 1)
    got = _run(M, grid, snaps, st0, groups)
    for k in ("id", "lon", "lat", "p", "up", "vp", "wp"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_host_snapshots_prefetched(M):
    """Snapshots in pinned host memory (copied ahead on a copy stream) give the device-snapshot run."""
    from paper_2211_12616_gb300.simulation import Simulation, periodic_snapshots
    grid = grid_2deg_20lev()
    modes = fourier_modes(5)
    snaps = [fourier_snapshot(grid, modes, h * DT_MET, device="cuda", as_numpy=False) for h in range(4)]
    host = [{k: v.cpu().pin_memory() for k, v in s.items()} for s in snaps]
    st0 = uniform_particles(20_000, grid.plev, 8)
    out = []
    for source in (snaps, host):
        ctx = M.Context(grid, M.MPTRAC_FP32)
        parts = M.Particles.from_numpy(st0)
        sim = Simulation(ctx, periodic_snapshots(source, DT_MET), DT_MET, parts, DT, M.DiffParams(), 4, 20)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            assert sim.run(0.0, 4 * DT_MET, stream=s) == 480
        torch.cuda.synchronize()
        got = parts.to_numpy()
        ctx.close()
        order = np.argsort(got["id"])
        out.append({k: v[order] for k, v in got.items()})
    for k in ("lon", "lat", "p", "up", "vp", "wp"):
        np.testing.assert_array_equal(out[1][k], out[0][k], err_msg=k)
