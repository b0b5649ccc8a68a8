"""Host-side scheduling logic of the Python layer (no GPU): the per-interval plan of a
batched run, the autotuner's candidate list and result cache, periodic snapshots."""
import json
from types import SimpleNamespace

import pytest

from paper_2211_12616_gb300.autotune import autotune, candidates
from paper_2211_12616_gb300.batch import BatchedRun
from paper_2211_12616_gb300.simulation import periodic_snapshots

DT, DT_MET = 180.0, 21600.0


def _plan(t_end, sort_every, dt=DT, dt_met=DT_MET):
    return BatchedRun._plan(SimpleNamespace(dt_met=dt_met, dt=dt, sort_every=sort_every), 0.0, t_end)


@pytest.mark.parametrize("sort_every", [10, 50, 120, 500])
def test_batch_plan_covers_every_step_once(sort_every):
    plan = _plan(72 * 3600.0, sort_every)
    assert len(plan) == 12
    steps_per_iv = int(DT_MET / DT)
    step = 0
    for iv, (loads, blocks) in enumerate(plan):
        ta = iv * DT_MET
        assert sum(cnt for _, _, cnt in blocks) == steps_per_iv
        assert all(cnt <= sort_every for _, _, cnt in blocks)
        for t, step0, cnt in blocks:
            assert step0 == step                       # global step index runs on without gaps
            assert t == pytest.approx(ta + (step0 - iv * steps_per_iv) * DT)
            step += cnt
    assert step == 12 * steps_per_iv


def test_batch_plan_loads_each_snapshot_once_into_the_free_slot():
    plan = _plan(72 * 3600.0, 120)
    held = {}
    for iv, (loads, _) in enumerate(plan):
        ta, tb = iv * DT_MET, (iv + 1) * DT_MET
        if iv == 0:
            assert sorted(t for _, t in loads) == [ta, tb]
        else:
            assert loads == [(loads[0][0], tb)]        # only the later snapshot is new
            assert held[loads[0][0]] != ta             # it never replaces the one still in use
        for slot, t in loads:
            assert slot in (0, 1)
            held[slot] = t
        assert sorted(held.values()) == [ta, tb]


def test_batch_plan_rejects_a_fractional_interval():
    with pytest.raises(ValueError):
        _plan(24 * 3600.0, 20, dt=7000.0)


def test_candidates_are_the_full_product():
    c = candidates()
    # block schedules: 1, 2 or 4 particles per thread, or one persistent wave
    assert len(c) == 7 * 4 * 5
    assert {(x["variant"], x["persistent"], x["per_thread"], x["sort_every"]) for x in c} == {
        (v, p, k, s) for v in range(7) for (p, k) in ((False, 1), (False, 2), (False, 4), (True, 1))
        for s in (5, 10, 20, 40, 120)}
    g = candidates(variants=(2,), persistent=(False,), sort_every=(20,), groups=(1, 2, 3), per_thread=(1,))
    assert [x["groups"] for x in g] == [1, 2, 3]


def test_autotune_returns_a_cached_result_without_running(tmp_path):
    best = {"variant": 2, "persistent": False, "sort_every": 20, "groups": 2}
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"gb300/1deg": {"best": best, "timings": {"x": 1.0}}}))

    def make_run(cfg):
        raise AssertionError("a cached key must not be timed")
    got, timings = autotune(make_run, lambda: None, candidates(), None, cache_path=str(path),
                            cache_key="gb300/1deg")
    assert got == best and timings == {"x": 1.0}


def test_periodic_snapshots_wrap_and_round():
    snaps = [{"u": i, "v": 10 + i, "w": 20 + i} for i in range(4)]
    at = periodic_snapshots(snaps, DT_MET)
    assert at(0.0) == (0, 10, 20)
    assert at(3 * DT_MET) == (3, 13, 23)
    assert at(4 * DT_MET) == (0, 10, 20)            # 24 h period
    assert at(5 * DT_MET - 1e-6) == (1, 11, 21)     # rounding to the nearest snapshot time
    assert at(-DT_MET) == (3, 13, 23)
