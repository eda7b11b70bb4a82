"""The serving scheduler's host logic (paper_2003_08374_gb300/serve.py) on the CPU, with
the library replaced by a fake that records what the scheduler asks of it: requests run
exactly their own step counts, admission respects the memory budget and the slot limit,
a request too large for an idle device is rejected, a diverged member is retired while
the others continue, and a round whose solve did not converge is counted."""
import types

import pytest

from paper_2003_08374_gb300 import mdbs, serve


class FakeSim:
    def __init__(self, case):
        self.case = case
        self.steps = 0
        self.closed = False
        self.diverged = False

    def set_stream(self, h):
        pass

    def stats(self):
        bad = float("nan") if self.diverged else 1.0
        return {"steps": self.steps, "mass": bad, "alpha_min": 0.0 if not self.diverged else bad,
                "alpha_max": 1.0, "cg_iters": [3, 2]}

    def fields(self):
        return {"steps": self.steps}

    def close(self):
        self.closed = True


class FakeBatch:
    log = []        # (round index, member names, steps) of every batch step
    fail = {}       # round index -> ("diverged", name) or ("not_converged", None)

    def __init__(self, sims):
        self.sims = list(sims)

    def set_stream(self, h):
        pass

    def add(self, sim):
        self.sims.append(sim)

    def remove(self, sim):
        self.sims.remove(sim)

    def step(self, n):
        r = len(FakeBatch.log)
        FakeBatch.log.append((r, sorted(s.case.name for s in self.sims), n))
        for s in self.sims:
            s.steps += n
        kind = FakeBatch.fail.get(r)
        if kind and kind[0] == "diverged":
            for s in self.sims:
                if s.case.name == kind[1]:
                    s.diverged = True
            raise mdbs.MdbsError(mdbs.ERR_DIVERGED, "non-finite field")
        if kind and kind[0] == "not_converged":
            raise mdbs.MdbsError(mdbs.ERR_NOT_CONVERGED, "max_cg reached")

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    FakeBatch.log = []
    FakeBatch.fail = {}
    monkeypatch.setattr(mdbs, "Simulation", FakeSim)
    monkeypatch.setattr(mdbs, "Batch", FakeBatch)
    monkeypatch.setattr(mdbs, "bytes_required", lambda case, precision=None: case.bytes)
    return FakeBatch


def case(name, cells, nbytes):
    return types.SimpleNamespace(name=name, cells=cells, bytes=nbytes)


def clock_of(times):
    """A clock that advances by the given increments, then stays."""
    state = {"t": 0.0, "i": 0}

    def clock():
        if state["i"] < len(times):
            state["t"] += times[state["i"]]
            state["i"] += 1
        return state["t"]
    return clock


def test_every_request_runs_exactly_its_steps_and_releases_its_memory(fake):
    reqs = [serve.Request(rid=i, arrival=0.0, case=case("r%d" % i, 1000 * (i + 1), 10), steps=s)
            for i, s in enumerate((7, 25, 13))]
    srv = serve.Server(max_active=8, round_steps=10, reserve_bytes=0, free_bytes_fn=lambda: 1000)
    out = srv.run(reqs, clock=clock_of([0.0] + [0.01] * 100))
    assert out["completed"] == 3 and out["rejected"] == 0 and out["failed"] == 0
    assert all(r.stats["steps"] == r.steps for r in reqs)
    # a round never passes a member's remaining steps (round limit 10): all advance 7 (r0
    # done), then r1 and r2 6 (r2 done at 13), then r1 alone 10 and 2 (25)
    assert [n for _, _, n in fake.log] == [7, 6, 10, 2]
    assert [names for _, names, _ in fake.log] == [["r0", "r1", "r2"], ["r1", "r2"], ["r1"], ["r1"]]
    assert out["served_cell_steps_per_s"] is not None
    assert srv.cell_steps == sum(r.case.cells * r.steps for r in reqs)


def test_admission_respects_memory_and_slots(fake):
    # budget 25 bytes: two requests of 10 fit, the third waits for one to finish
    reqs = [serve.Request(rid=i, arrival=0.0, case=case("m%d" % i, 100, 10), steps=5 * (i + 1)) for i in range(3)]
    srv = serve.Server(max_active=8, round_steps=100, reserve_bytes=0, free_bytes_fn=lambda: 25)
    out = srv.run(reqs, clock=clock_of([0.0] + [0.01] * 100))
    assert out["completed"] == 3
    first = fake.log[0][1]
    assert first == ["m0", "m1"]  # m2 waits: 3 x 10 > 25
    assert any("m2" in names for _, names, _ in fake.log[1:])
    assert out["peak_active"] == 2
    # the slot limit binds the same way
    fake.log.clear()
    srv = serve.Server(max_active=1, round_steps=100, reserve_bytes=0, free_bytes_fn=lambda: 10 ** 9)
    reqs = [serve.Request(rid=i, arrival=0.0, case=case("s%d" % i, 100, 10), steps=3) for i in range(3)]
    out = srv.run(reqs, clock=clock_of([0.0] + [0.01] * 100))
    assert out["completed"] == 3 and out["peak_active"] == 1
    assert all(len(names) == 1 for _, names, _ in fake.log)


def test_request_larger_than_an_idle_device_is_rejected(fake):
    reqs = [serve.Request(rid=0, arrival=0.0, case=case("huge", 10, 500), steps=4),
            serve.Request(rid=1, arrival=0.0, case=case("small", 10, 5), steps=4)]
    srv = serve.Server(max_active=8, round_steps=10, reserve_bytes=0, free_bytes_fn=lambda: 100)
    out = srv.run(reqs, clock=clock_of([0.0] + [0.01] * 100))
    assert reqs[0].rejected and out["rejected"] == 1
    assert out["completed"] == 1 and reqs[1].stats["steps"] == 4


def test_diverged_member_is_retired_and_the_others_continue(fake):
    fake.fail[0] = ("diverged", "bad")
    reqs = [serve.Request(rid=0, arrival=0.0, case=case("bad", 10, 1), steps=20),
            serve.Request(rid=1, arrival=0.0, case=case("good", 10, 1), steps=20)]
    srv = serve.Server(max_active=8, round_steps=10, reserve_bytes=0, free_bytes_fn=lambda: 100)
    out = srv.run(reqs, clock=clock_of([0.0] + [0.01] * 100))
    assert reqs[0].error == "diverged" and reqs[0].finished is None
    assert out["failed"] == 1 and out["completed"] == 1
    assert reqs[1].stats["steps"] == 20
    assert fake.log[1][1] == ["good"]


def test_unconverged_round_is_counted_and_the_run_continues(fake):
    fake.fail[0] = ("not_converged", None)
    reqs = [serve.Request(rid=0, arrival=0.0, case=case("a", 10, 1), steps=15)]
    srv = serve.Server(max_active=8, round_steps=10, reserve_bytes=0, free_bytes_fn=lambda: 100)
    out = srv.run(reqs, clock=clock_of([0.0] + [0.01] * 100))
    assert out["rounds_with_unconverged_solves"] == 1
    assert out["completed"] == 1 and reqs[0].stats["steps"] == 15
