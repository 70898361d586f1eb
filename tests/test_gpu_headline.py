"""Parity at the sizes the throughput is quoted on.

* The 2^24-particle piston tube (8 x 1 x 1, lambda = 0.02, u_p = 2, seed 2): the
  binary64 GPU path equals the oracle's first two steps (candidate pairs, partners,
  per-step counts, the whole state bit for bit), and the guarded binary32 path, in
  the launch configurations the benchmark's autotuner chooses between, equals the
  binary64 path for ten steps (sorted candidate-pair lists, partners, counts and the
  state in every step).  Paper, Sec. 2 ("Initial Simulation Setup"): the three
  criteria and the closest collision partner fix the candidate list and the pairs,
  so a faster pre-test may change the work, never the list.
* The 2^20-particle piston tube (the configuration the Rankine-Hugoniot pin uses) for
  100 steps, past the formation of the shock: trajectory, counts and profiles.
* The batched ensemble: 32 runs with N log-spaced over [2^12, 2^18] (equilibrium
  boxes and piston tubes), stepped as one group, each equal to the oracle.
* The spherical blast at 2^17 particles for 100 steps (its expansion).
"""
import math

import numpy as np
import pytest

import kmc_inputs as ki
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1310_3437_gb300 as kmc  # noqa: E402

FP64 = kmc.KMC_FP64
FP32 = kmc.KMC_GUARDED_FP32


def _sim(setup, arrays, precision, **knobs):
    p = kmc.params_from_setup(setup, precision=precision, **knobs)
    return kmc.Simulation(p, arrays)


def _device_state(sim, buf):
    """The state (52 n bytes: six binary64 components, then the last partners) gathered
    into a device buffer, compared on the device.  The gather runs on the simulation's
    stream (its own stream when created without one): wait for it before torch reads
    the buffer on another stream."""
    sim.state_device(buf)
    torch.cuda.synchronize()
    return buf


def _assert_counts_equal(a, b, what):
    assert len(a) == len(b), what
    for x, y in zip(a, b):
        assert (x["step"], x["collisions"], x["edges"], x["round_pairs"]) == \
               (y["step"], y["collisions"], y["edges"], y["round_pairs"]), (what, x, y)


def _assert_state_equals_oracle(sim, st, what):
    arrays, last = sim.state()
    for k in range(6):
        a, b = arrays[k].view(np.uint64), st.a[k].view(np.uint64)
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError(f"{what}: component {k}, {len(bad)} particles differ, "
                                 f"first ids {bad[:5]}")
    assert np.array_equal(last, st.last), what


# the launch configurations the benchmark's autotuner picks from for this workload
# (search kernel, stencil): the per-step automatic choice, the row search, the
# 125-cell stencil
HEADLINE_FP32_KNOBS = [
    {"search_kernel": 0, "stencil": 1},
    {"search_kernel": 3, "stencil": 1},
    {"search_kernel": 0, "stencil": 2},
]


def test_headline_tube_2e24_binary32_equals_binary64_and_the_oracle():
    n = 1 << 24
    s = ki.piston_setup(n=n, seed=2, profile_bins=256, profile_every=100)
    arrays = ki.initial_state(s)
    dev = [torch.from_numpy(a).cuda() for a in arrays]
    ref = _sim(s, dev, FP64)
    alts = [_sim(s, dev, FP32, **kn) for kn in HEADLINE_FP32_KNOBS]
    del dev
    bref = torch.empty(52 * n, dtype=torch.uint8, device="cuda")
    balt = torch.empty_like(bref)
    st = oracle.State(arrays)
    del arrays
    steps, oracle_steps = 10, 2
    for step in range(steps):
        if step < oracle_steps:
            pi, pj, _, _ = oracle.candidate_pairs(s, st)
            ocounts, opartner, _ = oracle.step(s, st, step)
        ref.step(1).sync()
        e_ref, p_ref, c_ref = ref.edges(), ref.partners(), ref.counts()
        assert len(c_ref) == 1 and c_ref[0]["step"] == step
        assert c_ref[0]["edges"] == e_ref.shape[0] > 100000, "a realistic candidate list"
        if step < oracle_steps:
            want = np.stack([pi, pj], axis=1)
            assert np.array_equal(e_ref, want), f"binary64 candidate pairs, step {step}"
            assert np.array_equal(p_ref, opartner), f"binary64 partners, step {step}"
            _assert_counts_equal(c_ref, [ocounts], f"binary64 counts, step {step}")
            _assert_state_equals_oracle(ref, st, f"binary64 state after step {step}")
        _device_state(ref, bref)
        for kn, alt in zip(HEADLINE_FP32_KNOBS, alts):
            alt.step(1).sync()
            what = f"binary32 {kn}, step {step}"
            assert np.array_equal(alt.edges(), e_ref), what + ": candidate pairs"
            assert np.array_equal(alt.partners(), p_ref), what + ": partners"
            _assert_counts_equal(alt.counts(), c_ref, what)
            _device_state(alt, balt)
            assert torch.equal(balt, bref), what + ": state"
    for sim in [ref] + alts:
        sim.close()


def test_config1_tube_2e20_past_shock_formation_bit_exact():
    """100 steps of the 2^20-particle tube (about eight collision times: the piston has
    driven a shock into the gas), both precisions; profiles every 25 steps."""
    s = ki.piston_setup(n=1 << 20, seed=2, profile_bins=256, profile_every=25)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    steps = 100
    oc, oprof = oracle.run(s, st, 0, steps)
    # the piston has compressed the gas: the profile's densest bin is well above the
    # initial density (2^20 / 256 particles per bin)
    assert oprof[-1][:, 0].max() > 1.8 * (1 << 20) / 256
    for prec in (FP64, FP32):
        sim = _sim(s, arrays, prec).step(steps).sync()
        got = sim.counts()
        _assert_counts_equal(got, oc, f"precision {prec}")
        assert [(g["absorbed"], g["live"]) for g in got] == [(o["absorbed"], o["live"]) for o in oc]
        _assert_state_equals_oracle(sim, st, f"precision {prec}")
        gprof = sim.profiles()
        assert gprof.shape == oprof.shape
        assert np.array_equal(gprof[:, :, 0], oprof[:, :, 0])
        # the oracle's id-order binary64 sums: |error| <= (count + 2) u sum|terms|
        u = 2.0 ** -53
        cnt = oprof[:, :, 0]
        for q in range(1, 7):
            sq = oprof[:, :, 4 + (q - 1) % 3]
            abs_sum = np.sqrt(np.maximum(cnt * sq, 0)) if q <= 3 else sq
            tol = (cnt + 2) * u * abs_sum + cnt * 2.0 ** -64 + 2 * u * np.abs(oprof[:, :, q])
            assert np.all(np.abs(gprof[:, :, q] - oprof[:, :, q]) <= tol), q
        sim.close()


def _ensemble_runs(count=32, lo=1 << 12, hi=1 << 18):
    """count runs with N log-spaced over [lo, hi] (the ensemble's range, both ends
    included), even index an equilibrium box with n sigma fixed, odd index a piston
    tube with u_p in [1, 3]; the oracle's cost of a dense box grows as N^2, so the
    step count shrinks with N (at least 2 steps)."""
    out = []
    for k in range(count):
        n = int(round(lo * (hi / lo) ** (k / (count - 1))))
        if k % 2 == 0:
            steps = max(2, min(25, int(25 * (1 << 14) ** 2 / n ** 2)))
            s = ki.equilibrium_setup(n=n, seed=1000 + k, d0=0.02 * math.sqrt(4096.0 / n),
                                     steps=steps)
        else:
            rng = np.random.default_rng(1000 + k)
            s = ki.piston_setup(n=n, seed=1000 + k, u_p=float(rng.uniform(1.0, 3.0)),
                                steps=25, profile_bins=0, profile_every=0)
        out.append(s)
    return out


def test_ensemble_32_runs_spanning_2e12_to_2e18_as_one_group():
    setups = _ensemble_runs()
    assert setups[0].n == 1 << 12 and setups[-1].n == 1 << 18
    arrays = [ki.initial_state(q) for q in setups]
    want = []
    for q, a in zip(setups, arrays):
        st = oracle.State(a)
        oc, _ = oracle.run(q, st, 0, q.steps)
        want.append((oc, st))
    for precision in (FP32, FP64):
        sims = [_sim(q, a, precision) for q, a in zip(setups, arrays)]
        g = kmc.Group(sims)
        for q, sim in zip(setups, sims):
            g.budget(sim, q.steps)
        g.step(max(q.steps for q in setups))
        g.sync()
        for q, sim, (oc, st) in zip(setups, sims, want):
            what = f"{q.name}, precision {precision}"
            assert g.steps_left(sim) == 0, what
            _assert_counts_equal(sim.counts(), oc, what)
            _assert_state_equals_oracle(sim, st, what)
        g.close()
        for sim in sims:
            sim.close()


def test_spherical_blast_2e17_for_100_steps_bit_exact():
    """The spherical blast (hot ball at 8x density and 100x temperature, background mean
    free path 0.005) at 2^17 particles for 100 steps: the hot ball's particles travel
    about four ball radii, so the run covers the blast's expansion and the speed split
    changes its threshold as the fast tail thins out.  The full size (2^27) is out of
    the oracle's reach (its cells are sized for the fastest particle: ~10^13 pair tests
    per step); the GPU runs it in the benchmark."""
    s = ki.blast_setup(n=1 << 17, seed=3, steps=100)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    oc, _ = oracle.run(s, st, 0, 100)
    assert sum(c["collisions"] for c in oc) > 500000
    for prec in (FP32, FP64):
        sim = _sim(s, arrays, prec).step(100).sync()
        got = sim.counts()
        _assert_counts_equal(got, oc, f"blast, precision {prec}")
        assert sum(c["fast_tests"] for c in got) > 0, "the speed split ran"
        _assert_state_equals_oracle(sim, st, f"blast, precision {prec}")
        sim.close()
