"""The serving loop's host-side scheduling, with stand-ins for the simulations and the
group (no GPU): admission in arrival order while the device footprint fits the
budget, bursts that never run past the end of the live request closest to its end,
every request retired with exactly its steps, memory returned on retirement, and a
request larger than the budget refused up front."""
from types import SimpleNamespace

import pytest

from paper_1310_3437_gb300 import serve


class FakeSim:
    def __init__(self, params):
        self.n = params.n
        self.steps_run = 0
        self.closed = False

    def state(self):
        return ("state", self.n, self.steps_run)

    def counts(self):
        return [{"step": k} for k in range(self.steps_run)]

    def close(self):
        self.closed = True


class FakeGroup:
    """Steps every member with budget left; records each burst's length against the
    smallest budget left among the live members."""
    log = []

    def __init__(self, sims, stream=None):
        self.left = {}
        for s in sims:
            self.left[s] = 0

    def add(self, sim):
        assert sim not in self.left
        self.left[sim] = 0

    def remove(self, sim):
        assert self.left[sim] == 0
        del self.left[sim]

    def budget(self, sim, steps):
        self.left[sim] += steps

    def step(self, k):
        live = [b for b in self.left.values() if b > 0]
        FakeGroup.log.append((k, min(live) if live else 0))
        for s in self.left:
            d = min(k, self.left[s])
            self.left[s] -= d
            s.steps_run += d

    def sync(self):
        pass

    def steps_left(self, sim):
        return self.left[sim]

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    FakeGroup.log = []
    monkeypatch.setattr(serve, "Simulation", lambda params, arrays=None, init=None, stream=None:
                        FakeSim(params))
    monkeypatch.setattr(serve, "Group", FakeGroup)
    monkeypatch.setattr(serve, "params_from_setup",
                        lambda setup, precision=None, history_cap=0: SimpleNamespace(n=setup.n))
    monkeypatch.setattr(serve, "sim_bytes_required", lambda params: 100 * params.n)
    return FakeGroup


def _requests():
    # (n, steps, arrival): sizes and lengths uneven, arrivals within a few ms
    spec = [(1000, 40, 0.000), (3000, 7, 0.001), (500, 100, 0.001), (4000, 25, 0.002),
            (2000, 3, 0.002), (3500, 60, 0.003), (800, 16, 0.004), (2500, 33, 0.004),
            (1200, 1, 0.005), (3900, 50, 0.006)]
    return [serve.Request(rid=i, setup=SimpleNamespace(n=n), steps=st, arrival=t, arrays=[])
            for i, (n, st, t) in enumerate(spec)]


def test_every_request_runs_exactly_its_steps_within_the_budget(fakes, monkeypatch):
    budget = 100 * 7000  # room for only a few requests at once
    srv = serve.Server(budget_bytes=budget, burst_steps=16)
    peak = {"in_use": 0, "order": []}
    admit = serve.Server._admit

    def watched_admit(self, req, now):
        admit(self, req, now)
        peak["in_use"] = max(peak["in_use"], self.in_use)
        peak["order"].append(req.rid)

    monkeypatch.setattr(serve.Server, "_admit", watched_admit)
    reqs = _requests()
    done, wall = srv.run(reqs)
    assert sorted(r.rid for r in done) == list(range(len(reqs)))
    for r in done:
        assert len(r.counts) == r.steps                 # exactly its steps, no more
        assert r.state == ("state", r.setup.n, r.steps)
        assert r.finished >= r.admitted >= r.arrival
    assert peak["in_use"] <= budget
    assert srv.in_use == 0 and not srv.live            # all memory returned
    # admission in arrival order (ties by id, as sorted)
    assert peak["order"] == [r.rid for r in sorted(reqs, key=lambda r: r.arrival)]
    # no burst runs past the end of the live request closest to its end, none exceeds 16
    for k, smallest in fakes.log:
        assert 1 <= k <= 16 and k <= smallest
    assert sum(r.setup.n * r.steps for r in done) == srv.particle_steps


def test_a_request_above_the_budget_is_refused(fakes):
    srv = serve.Server(budget_bytes=100 * 999)
    with pytest.raises(ValueError):
        srv.run([serve.Request(rid=0, setup=SimpleNamespace(n=1000), steps=5, arrival=0.0,
                               arrays=[])])


def test_summary_of_the_latencies(fakes):
    srv = serve.Server(budget_bytes=100 * 50000)
    done, wall = srv.run(_requests())
    s = serve.summarize(done, wall)
    assert s["requests"] == 10
    assert s["particle_steps"] == sum(r.setup.n * r.steps for r in done)
    assert 0 <= s["p50_latency_s"] <= s["p99_latency_s"]
