"""Serving loop: requests admitted under an HBM budget and stepped together give the
same result as each request run alone (bit-exact final state and per-step counts)."""
import numpy as np
import pytest

import kmc_inputs as ki

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1310_3437_gb300 as kmc  # noqa: E402
from paper_1310_3437_gb300.serve import Request, Server, summarize  # noqa: E402


def _stream(count, seed=7):
    setups = ki.serving_requests(count, master_seed=seed, n_lo=1 << 10, n_hi=1 << 13,
                                 steps_lo=5, steps_hi=40)
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(0.01, size=count))
    return [Request(rid=k, setup=s, steps=s.steps, arrival=float(t[k]),
                    arrays=ki.initial_state(s)) for k, s in enumerate(setups)]


@pytest.mark.parametrize("precision", [kmc.KMC_GUARDED_FP32, kmc.KMC_FP64])
def test_results_in_the_mix_equal_results_alone(precision):
    reqs = _stream(14)
    for r in reqs:
        r.precision = precision
    # a budget of about three requests forces queueing and turnover
    sizes = [kmc.sim_bytes_required(kmc.params_from_setup(r.setup, precision=precision,
                                                          history_cap=max(64, r.steps + 8)))
             for r in reqs]
    server = Server(budget_bytes=3.2 * max(sizes), burst_steps=4)
    done, wall = server.run(reqs)
    assert len(done) == len(reqs)
    assert max(r.bytes for r in reqs) <= server.budget
    summary = summarize(done, wall)
    assert summary["p99_latency_s"] >= summary["p50_latency_s"] > 0
    for r in done:
        alone = kmc.Simulation(kmc.params_from_setup(r.setup, precision=precision),
                               ki.initial_state(r.setup))
        alone.step(r.steps).sync()
        arrays, last = alone.state()
        got, glast = r.state
        for a, b in zip(arrays, got):
            assert np.array_equal(a, b), f"request {r.rid}"
        assert np.array_equal(last, glast)
        ca = alone.counts()
        assert [c["collisions"] for c in ca] == [c["collisions"] for c in r.counts]
        assert len(r.counts) == r.steps
        alone.close()


def test_admission_never_exceeds_the_budget():
    reqs = _stream(10, seed=11)
    sizes = [kmc.sim_bytes_required(kmc.params_from_setup(r.setup, precision=r.precision,
                                                          history_cap=max(64, r.steps + 8)))
             for r in reqs]
    budget = 1.5 * max(sizes)
    server = Server(budget_bytes=budget, burst_steps=8, keep_state=False)
    peak = {"v": 0}
    orig = server._admit

    def admit(req, now):
        orig(req, now)
        peak["v"] = max(peak["v"], server.in_use)

    server._admit = admit
    done, _ = server.run(reqs)
    assert len(done) == 10
    assert peak["v"] <= budget


def test_requests_with_device_drawn_states_equal_the_oracle_run():
    """Requests that carry an init descriptor (state drawn on the device at
    admission) end in the oracle's state for the same descriptor."""
    import oracle
    setups = ki.serving_requests(6, master_seed=13, n_lo=1 << 10, n_hi=1 << 12,
                                 steps_lo=5, steps_hi=20)
    reqs = [Request(rid=k, setup=s, steps=s.steps, arrival=0.001 * k, init=ki.init_spec(s))
            for k, s in enumerate(setups)]
    server = Server(budget_bytes=64e9, burst_steps=4)
    done, _ = server.run(reqs)
    for r in done:
        st = oracle.State(oracle.init_particles(r.setup, ki.init_spec(r.setup)))
        oracle.run(r.setup, st, 0, r.steps)
        got, glast = r.state
        for a, b in zip(st.a, got):
            assert np.array_equal(a, b), f"request {r.rid}"
        assert np.array_equal(st.last, glast)
