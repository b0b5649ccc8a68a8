"""The schedule Simulation.run issues (no GPU): CUDA streams and events are replaced by
recording fakes, the context by a recorder of the ABI calls.  Checked: the ring of three met
slots (snapshot k in slot k mod 3, each loaded once, a slot overwritten only after every group
has finished the interval that last read it), sorts and fused steps covering every step of
every group once, hand-off sorts between blocks and none after the last one."""
import contextlib
from types import SimpleNamespace

import pytest
import torch

import paper_2211_12616_gb300.simulation as simmod

DT, DT_MET = 180.0, 21600.0


class FakeStream:
    log = None

    def __init__(self, device=None, priority=0):
        self.name = f"s{len(FakeStream.log['streams'])}"
        FakeStream.log["streams"].append(self)

    @staticmethod
    def priority_range():
        return 0, -1

    def wait_stream(self, other):
        FakeStream.log["ops"].append(("wait_stream", self.name, other.name))

    def wait_event(self, ev):
        FakeStream.log["ops"].append(("wait_event", self.name, ev.id))


class FakeEvent:
    count = 0

    def __init__(self, **kw):
        FakeEvent.count += 1
        self.id = FakeEvent.count

    def record(self, stream):
        FakeStream.log["ops"].append(("record", stream.name, self.id))


class FakeParticles:
    def __init__(self, n, a=0):
        self.n, self.a = n, a
        self.lon = SimpleNamespace(device="cpu")

    def view(self, a, b):
        return FakeParticles(b - a, self.a + a)


class FakeCtx:
    def __init__(self, log):
        self.log = log

    def sort_workspace_bytes(self, n):
        return 0

    def load_met(self, slot, t, *fields, stream=None):
        self.log["ops"].append(("load", stream.name, slot, t))

    def sort(self, parts, ws, stream=None):
        self.log["ops"].append(("sort", stream.name, parts.a))

    def sort_handoff(self, parts, ws, stream=None):
        self.log["ops"].append(("sort_handoff", stream.name, parts.a))

    def step(self, parts, t, dt, prm, seed, step0, n, stream=None):
        self.log["ops"].append(("step", stream.name, parts.a, t, step0, n))

    def step_handoff(self, parts, t, dt, prm, seed, step0, n, ws, stream=None):
        self.log["ops"].append(("step_handoff", stream.name, parts.a, t, step0, n))


@pytest.fixture
def fakes(monkeypatch):
    log = {"streams": [], "ops": []}
    FakeStream.log = log
    main = FakeStream()
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda dev=None: main)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    return log, main


@pytest.mark.parametrize("groups", [1, 2, 3])
@pytest.mark.parametrize("hours", [6, 12, 24, 48])
def test_ring_sorts_and_steps(fakes, groups, hours):
    log, main = fakes
    n = 1000
    sim = simmod.Simulation(FakeCtx(log), lambda t: (t, t, t), DT_MET, FakeParticles(n), DT, None, 7,
                            sort_every=20, groups=groups)
    nsteps = sim.run(0.0, hours * 3600.0)
    n_iv = hours // 6
    assert nsteps == n_iv * 120
    ops = log["ops"]
    loads = [o for o in ops if o[0] == "load"]
    # every snapshot of the run once, snapshot k in slot k mod 3
    assert [o[3] for o in loads] == [k * DT_MET for k in range(n_iv + 1)]
    assert [o[2] for o in loads] == [k % 3 for k in range(n_iv + 1)]
    assert loads[0][1] == loads[1][1] == main.name          # the first two in stream order
    # a snapshot k >= 3 overwrites snapshot k - 3, read last by interval k - 3: its load comes
    # after every group's last step of that interval, and its stream waits for each group stream
    step_ops = [i for i, o in enumerate(ops) if o[0] in ("step", "step_handoff")]
    for k in range(3, n_iv + 1):
        i_load = ops.index(loads[k])
        last_iv = [i for i in step_ops if ops[i][4] < (k - 2) * 120]
        assert max(last_iv) < i_load
        waits = [o for o in ops[max(last_iv):i_load] if o[0] == "wait_stream" and o[1] == loads[k][1]]
        assert len({o[2] for o in waits}) == groups
    # steps: per group, blocks of 20 covering [0, nsteps) once; hand-off on all but the last
    for g in range(groups):
        a = round(g * n / groups)
        mine = [ops[i] for i in step_ops if ops[i][2] == a]
        assert [o[4] for o in mine] == list(range(0, nsteps, 20))
        assert all(o[5] == 20 for o in mine)
        assert all(o[3] == pytest.approx(o[4] * DT) for o in mine)
        assert [o[0] for o in mine] == ["step_handoff"] * (len(mine) - 1) + ["step"]
        sorts = [o for o in ops if o[0] in ("sort", "sort_handoff") and o[2] == a]
        assert [o[0] for o in sorts] == ["sort"] + ["sort_handoff"] * (len(mine) - 1)


def test_zero_length_run_issues_nothing(fakes):
    log, _ = fakes
    sim = simmod.Simulation(FakeCtx(log), lambda t: (t, t, t), DT_MET, FakeParticles(10), DT, None, 7)
    assert sim.run(0.0, 0.0) == 0
    assert not [o for o in log["ops"] if o[0] in ("load", "sort", "step", "step_handoff")]


def test_fractional_interval_is_rejected(fakes):
    log, _ = fakes
    sim = simmod.Simulation(FakeCtx(log), lambda t: (t, t, t), DT_MET, FakeParticles(10), 7000.0, None, 7)
    with pytest.raises(ValueError):
        sim.run(0.0, DT_MET)
