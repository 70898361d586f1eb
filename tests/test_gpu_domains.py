"""Domain decomposition into x slabs (Sec. 4, "Hybrid Simulations") on one GPU.

The paper splits the space into equal domains along one axis, keeps a row of ghost
cells from each neighbour, synchronises the adaptive time step through the global
maximum speed, sends the collision partners found for ghost particles back to their
owners so that mutual choice across a cut is decided correctly, and migrates the
particles that crossed a cut.  The method's result does not depend on the split, so
a decomposed run must equal the single-domain run and the oracle bit for bit:
trajectories, per-step counts, candidate pairs and partners.
"""
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


def _dom(setup, arrays, precision, domains, **kw):
    p = kmc.params_from_setup(setup, precision=precision, **kw)
    p.profile_bins = 0
    p.profile_every = 0
    return kmc.Simulation(p, arrays, domains=domains)


def _assert_state(sim, st, what):
    arrays, last = sim.state()
    for k in range(6):
        a, b = arrays[k].view(np.uint64), st.a[k].view(np.uint64)
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError(f"{what}: component {k}, {len(bad)} differ, first ids {bad[:5]}")
    assert np.array_equal(last, st.last), what


def _assert_counts(got, want, what):
    assert len(got) == len(want), what
    for g, o in zip(got, want):
        assert (g["step"], g["collisions"], g["edges"], g["round_pairs"]) == \
               (o["step"], o["collisions"], o["edges"], o["round_pairs"]), (what, g, o)


def _tube(n=1 << 15, seed=61):
    return ki.piston_setup(n=n, seed=seed, box=(8.0, 0.25, 0.25), profile_bins=0,
                           profile_every=0)


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("domains", [1, 2, 3, 4])
def test_piston_tube_decomposed_equals_the_oracle(precision, domains):
    """50 steps of a piston tube cut into equal slabs along x: particles cross the
    cuts every step (thermal motion, and the piston sweeps the gas down through
    them)."""
    s = _tube()
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    oc, _ = oracle.run(s, st, 0, 50)
    sim = _dom(s, arrays, precision, domains)
    owner0 = np.minimum((arrays[0] * domains / 8.0).astype(int), domains - 1)
    sim.step(50).sync()
    _assert_counts(sim.counts(), oc, f"{domains} domains")
    _assert_state(sim, st, f"{domains} domains")
    owned, ghosts = sim.domains()
    assert owned.shape == (domains,) and owned.sum() == s.n
    if domains > 1:
        assert (ghosts > 0).all()
        moved = np.minimum((st.a[0] * domains / 8.0).astype(int), domains - 1) != owner0
        assert moved.sum() > 100, "particles crossed the cuts"
    assert sim.step_index() == 50
    sim.close()


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_decomposed_pair_lists_and_partners_every_step(precision):
    s = _tube(n=1 << 14, seed=62)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    sim = _dom(s, arrays, precision, 3)
    for step in range(8):
        pi, pj, _, _ = oracle.candidate_pairs(s, st)
        counts, partner, _ = oracle.step(s, st, step)
        sim.step(1).sync()
        assert np.array_equal(sim.edges(), np.stack([pi, pj], axis=1)), f"step {step}"
        assert np.array_equal(sim.partners(), partner), f"step {step}"
        _assert_counts(sim.counts(), [counts], f"step {step}")
    _assert_state(sim, st, "after 8 steps")
    assert sim.vmax() == np.sqrt(oracle.vmax2(st))
    sim.close()


@pytest.mark.parametrize("domains", [2, 5])
def test_periodic_x_wraps_ghosts_across_the_box_edge(domains):
    """An equilibrium box periodic in x: the first and the last domain are neighbours
    through the periodic boundary."""
    s = ki.equilibrium_setup(n=6000, seed=63)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    oc, _ = oracle.run(s, st, 0, 30)
    for precision in (FP64, FP32):
        sim = _dom(s, arrays, precision, domains).step(30).sync()
        _assert_counts(sim.counts(), oc, f"periodic, {domains} domains")
        _assert_state(sim, st, f"periodic, {domains} domains")
        sim.close()


def test_slabs_thinner_than_the_reach():
    """Sixteen slabs of a unit box whose reach d0 + 2 v_max dt spans several of them:
    ghosts come from beyond the neighbouring domains."""
    s = ki.equilibrium_setup(n=4000, seed=64, dt=0.02)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    oc, _ = oracle.run(s, st, 0, 20)
    sim = _dom(s, arrays, FP32, 16).step(20).sync()
    _assert_counts(sim.counts(), oc, "16 thin slabs")
    _assert_state(sim, st, "16 thin slabs")
    owned, ghosts = sim.domains()
    assert ghosts.sum() > 2 * owned.sum(), "each particle is a ghost in several domains"
    sim.close()


def test_planar_decomposition_and_resume():
    """A planar run (the paper's hybrid timing runs are two-dimensional) decomposed in
    four, stopped after 12 steps and resumed from its observed state: the same
    trajectory as one uninterrupted single-domain run."""
    s = ki.equal_speed_setup(n=5000, seed=65, planar=True)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    oc, _ = oracle.run(s, st, 0, 25)
    a = _dom(s, arrays, FP64, 4).step(12).sync()
    mid, last = a.state()
    b = kmc.Simulation(kmc.params_from_setup(s, precision=FP64, step0=12), mid, last=last,
                       domains=4)
    b.step(13).sync()
    _assert_counts(a.counts() + b.counts(), oc, "planar resumed")
    _assert_state(b, st, "planar resumed")
    a.close()
    b.close()


def test_decomposition_rejects_what_it_does_not_support():
    s = _tube(n=1000)
    arrays = ki.initial_state(s)
    with pytest.raises(kmc.KmcError):
        _dom(s, arrays, FP64, 0)
    with pytest.raises(kmc.KmcError):
        _dom(s, arrays, FP64, 65)
    p = kmc.params_from_setup(s, precision=FP64)
    p.profile_bins, p.profile_every = 16, 1
    with pytest.raises(kmc.KmcError):
        kmc.Simulation(p, arrays, domains=2)
    sim = _dom(s, arrays, FP64, 2)
    with pytest.raises(kmc.KmcError):
        kmc.Group([sim])
    sim.close()
