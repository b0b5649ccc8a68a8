"""Batched releases: release-aware sort, launch-schedule invariance, CUDA graphs, parity."""
import numpy as np
import pytest
import torch

from oracle import sort as osort
from oracle import transport as tr
from oracle.driver import run_schedule
from workloads import column_releases, fourier_modes, fourier_snapshot, grid_global

from _gpu_common import M, assert_positions_close, by_id  # noqa: F401

pytestmark = pytest.mark.gpu
DT, DT_MET = 180.0, 21600.0


@pytest.fixture(scope="module")
def case(M):
    grid = grid_global(120, 61, 30)
    modes = fourier_modes(4)
    snaps = [fourier_snapshot(grid, modes, h * DT_MET, device="cuda", as_numpy=False) for h in range(4)]
    rel = column_releases(16, seed=4, count_scale=4e-3, dur_min_h=2.0, dur_max_h=12.0)
    return grid, snaps, rel


def _at(snaps):
    from paper_2211_12616_gb300.simulation import periodic_snapshots
    return periodic_snapshots(snaps, DT_MET)


def test_sort_at_matches_oracle(M, case):
    """Times before every release, at the start, in the middle, and after every release has
    ended (nothing active: every key is the same and the order is kept); some particles
    carry a release index beyond the table (never active)."""
    grid, snaps, rel = case
    ctx = M.Context(grid)
    st = {k: v.copy() for k, v in rel.particles.items()}
    st["release"][::53] = len(rel.t_start) + 3
    ctx.set_releases(rel.t_start, rel.t_end)
    for t in (-3600.0, 0.0, 5 * 3600.0, 9 * 3600.0, 1e7):
        parts = M.Particles.from_numpy(st)
        ctx.sort_at(parts, t)
        torch.cuda.synchronize()
        perm = osort.sort_permutation_at(grid, st, t, (rel.t_start, rel.t_end))
        np.testing.assert_array_equal(parts.to_numpy()["id"], st["id"][perm])


def _run(M, case, cfg, graphs):
    from paper_2211_12616_gb300.batch import BatchedRun
    grid, snaps, rel = case
    ctx = M.Context(grid)
    parts = M.Particles.from_numpy(rel.particles)
    run = BatchedRun(ctx, _at(snaps), DT_MET, parts, rel.t_start, rel.t_end, DT, M.DiffParams(), 4,
                     sort_every=cfg["sort_every"], variant=cfg["variant"], persistent=cfg["persistent"],
                     per_thread=cfg.get("per_thread", 1))
    s = torch.cuda.Stream()
    if graphs:
        run.run_eager(0.0, 2 * DT_MET, stream=s)   # warm-up outside capture (occupancy queries)
        torch.cuda.synchronize()
        parts.copy_(M.Particles.from_numpy(rel.particles))
        run.capture(0.0, 2 * DT_MET, s)
        with torch.cuda.stream(s):
            run.replay()
    else:
        run.run_eager(0.0, 2 * DT_MET, stream=s)
    torch.cuda.synchronize()
    return by_id(parts.to_numpy())


def test_batched_run_parity_and_schedule_invariance(M, case):
    grid, snaps, rel = case
    base = _run(M, case, {"variant": 0, "persistent": False, "sort_every": 20}, graphs=False)
    host = [{k: v.cpu().numpy() for k, v in s.items()} for s in snaps]
    ref = run_schedule(grid, lambda t: host[int(round(t / DT_MET)) % 4], DT_MET, rel.particles, 0.0,
                       2 * DT_MET, DT, tr.DiffParams(), 4, windows=(rel.t_start, rel.t_end))
    ref = by_id(ref)
    assert_positions_close(base, ref, what="batched 12 h", lon_metric="arc")
    # particles of releases that ended early stopped at the same step as in the oracle
    ended = rel.t_end[rel.particles["release"][np.argsort(rel.particles["id"])]] < 2 * DT_MET
    assert ended.any()
    for cfg in ({"variant": 1, "persistent": True, "sort_every": 10},
                {"variant": 2, "persistent": True, "sort_every": 40},
                {"variant": 3, "persistent": False, "sort_every": 20},
                {"variant": 4, "persistent": True, "sort_every": 20},
                {"variant": 0, "persistent": True, "sort_every": 120},
                {"variant": 2, "persistent": False, "per_thread": 2, "sort_every": 5},
                {"variant": 3, "persistent": False, "per_thread": 4, "sort_every": 20},
                {"variant": 5, "persistent": False, "per_thread": 1, "sort_every": 40},
                {"variant": 6, "persistent": True, "sort_every": 10}):
        got = _run(M, case, cfg, graphs=True)
        for k in ("lon", "lat", "p", "up", "vp", "wp"):
            np.testing.assert_array_equal(got[k], base[k], err_msg=f"{cfg} {k}")


def test_autotuner_picks_a_candidate(M, case):
    from paper_2211_12616_gb300.autotune import autotune, candidates
    from paper_2211_12616_gb300.batch import BatchedRun
    grid, snaps, rel = case
    ctx = M.Context(grid)
    init = M.Particles.from_numpy(rel.particles)
    parts = init.clone()
    s = torch.cuda.Stream()

    def make(cfg):
        run = BatchedRun(ctx, _at(snaps), DT_MET, parts, rel.t_start, rel.t_end, DT, M.DiffParams(), 4,
                         sort_every=cfg["sort_every"], variant=cfg["variant"], persistent=cfg["persistent"],
                         per_thread=cfg["per_thread"])
        return lambda: run.run_eager(0.0, DT_MET, stream=s)

    cands = candidates(sort_every=(20, 120))
    best, timings = autotune(make, lambda: parts.copy_(init), cands, s, repeats=1)
    assert best in cands and len(timings) == len(cands)
    assert all(v > 0 for v in timings.values())
