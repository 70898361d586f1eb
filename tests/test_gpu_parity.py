"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Trajectories, candidate-pair lists, partners and per-step counts must be
bit-identical; profiles (order-free fixed-point sums on the GPU, id-order binary64
sums in the oracle) agree within the rounding bound of the oracle's summation.
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


def gpu_sim(setup, arrays, precision=FP64, stencil=1, cell_scale=1.0, last=None, step0=0,
            edge_cap=0, search_kernel=0, flags=0):
    p = kmc.params_from_setup(setup, precision=precision, stencil=stencil, cell_scale=cell_scale,
                              step0=step0, edge_cap=edge_cap, search_kernel=search_kernel)
    p.flags |= flags
    mixture = None
    if getattr(setup, "species", None) is not None:
        mixture = (setup.species, setup.masses, setup.radii)
    return kmc.Simulation(p, arrays, last=last, mixture=mixture)


def assert_same_state(sim, st: oracle.State):
    arrays, last = sim.state()
    for k in range(6):
        a, b = arrays[k], st.a[k]
        if not np.array_equal(a.view(np.uint64), b.view(np.uint64)):
            bad = np.nonzero(a.view(np.uint64) != b.view(np.uint64))[0]
            raise AssertionError(f"component {k}: {len(bad)} particles differ, first {bad[:5]}: "
                                 f"{a[bad[:3]]} vs {b[bad[:3]]}")
    assert np.array_equal(last, st.last)


def assert_same_counts(gpu_counts, or_counts):
    assert len(gpu_counts) == len(or_counts)
    for g, o in zip(gpu_counts, or_counts):
        assert g["step"] == o["step"]
        assert (g["collisions"], g["edges"], g["round_pairs"]) == \
               (o["collisions"], o["edges"], o["round_pairs"]), (g, o)
        assert (g["absorbed"], g["live"]) == (o["absorbed"], o["live"]), (g, o)


def run_both(setup, steps, precision=FP64, arrays=None, **kw):
    arrays = arrays if arrays is not None else ki.initial_state(setup)
    st = oracle.State(arrays)
    oc, oprof = oracle.run(setup, st, 0, steps)
    sim = gpu_sim(setup, arrays, precision=precision, **kw)
    sim.step(steps).sync()
    return sim, st, oc, oprof


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_equilibrium_box_4096_200_steps_bit_exact(precision):
    s = ki.equilibrium_setup(n=4096, seed=1)
    sim, st, oc, _ = run_both(s, 200, precision)
    assert_same_counts(sim.counts(), oc)
    assert_same_state(sim, st)
    assert sum(c["collisions"] for c in oc) > 20000


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_piston_tube_pair_lists_every_step(precision):
    s = ki.piston_setup(n=1 << 15, seed=2, box=(8.0, 0.25, 0.25), profile_bins=0, profile_every=0)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    sim = gpu_sim(s, arrays, precision=precision)
    for step in range(6):
        pi, pj, _, _ = oracle.candidate_pairs(s, st)
        counts, partner, _ = oracle.step(s, st, step)
        sim.step(1).sync()
        e = sim.edges()
        want = np.stack([pi, pj], axis=1)
        assert e.shape == want.shape and np.array_equal(e, want), f"step {step}"
        assert np.array_equal(sim.partners(), partner), f"step {step}"
    assert_same_state(sim, st)


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_piston_tube_trajectory_bit_exact(precision, kernel):
    s = ki.piston_setup(n=1 << 14, seed=3, box=(8.0, 0.125, 0.125), profile_bins=0,
                        profile_every=0)
    sim, st, oc, _ = run_both(s, 300, precision, search_kernel=kernel)
    assert_same_counts(sim.counts(), oc)
    assert_same_state(sim, st)


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("stencil,cell_scale,kernel", [
    (2, 1.0, 0), (1, 1.7, 0), (2, 2.3, 0), (1, 1.0, 1), (1, 1.0, 2), (2, 1.0, 1), (2, 1.0, 2),
    (1, 3.0, 2), (2, 4.0, 2), (1, 2.5, 1), (1, 1.0, 3), (2, 1.0, 3), (1, 2.0, 3), (2, 3.5, 3)])
def test_results_do_not_depend_on_grid_tuning(precision, stencil, cell_scale, kernel):
    """Cell size, stencil and search kernel (incl. cells above the per-warp staging
    capacity at cell_scale 3-4) change the work, never the result."""
    s = ki.equilibrium_setup(n=6000, seed=4)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    oracle.run(s, st, 0, 40)
    ref = gpu_sim(s, arrays, precision).step(40).sync()
    assert_same_state(ref, st)
    alt = gpu_sim(s, arrays, precision, stencil=stencil, cell_scale=cell_scale,
                  search_kernel=kernel).step(40).sync()
    a, la = ref.state()
    b, lb = alt.state()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(la, lb)
    assert [c["collisions"] for c in ref.counts()] == [c["collisions"] for c in alt.counts()]


def test_fp32_and_fp64_pair_lists_identical_with_many_near_threshold_pairs():
    """Velocities and positions on coarse lattices make many pairs sit exactly on or
    within a few ulps of the t* = 0, t* = dt and d_min = d0 thresholds."""
    rng = np.random.default_rng(5)
    n = 5000
    L = 1.0
    pos = [np.minimum(np.round(rng.random(n) * 64) / 64, np.nextafter(L, 0)) for _ in range(3)]
    vel = [np.round(rng.normal(0, 1, n) * 8) / 8 for _ in range(3)]
    s = ki.Setup(n=n, box=(L, L, L), bc=(0, 0, 0), d0=1 / 32, dt=1 / 16, seed=5,
                 name="equilibrium_lattice")
    st = oracle.State(pos + vel)
    pi, pj, _, _ = oracle.candidate_pairs(s, st)
    for prec in (FP64, FP32):
        for kern in (1, 2, 3):
            sim = gpu_sim(s, pos + vel, prec, search_kernel=kern).step(1).sync()
            e = sim.edges()
            assert np.array_equal(e, np.stack([pi, pj], axis=1))


def test_edge_cases():
    # one particle
    s = ki.equilibrium_setup(n=1, seed=1)
    sim, st, oc, _ = run_both(s, 5)
    assert_same_state(sim, st)
    # a head-on pair
    s = ki.Setup(n=2, box=(1.0, 1.0, 1.0), bc=(0, 0, 0), d0=0.05, dt=0.1, seed=9,
                 name="equilibrium_pair")
    arrays = [np.array([0.40, 0.45]), np.array([0.5, 0.51]), np.array([0.5, 0.5]),
              np.array([0.3, -0.3]), np.array([0.0, 0.0]), np.array([0.0, 0.0])]
    for prec in (FP64, FP32):
        sim, st, oc, _ = run_both(s, 3, prec, arrays=arrays)
        assert oc[0]["collisions"] == 1
        assert_same_counts(sim.counts(), oc)
        assert_same_state(sim, st)
    # thin periodic slab (y and z collapse to one cell), particles on the faces
    rng = np.random.default_rng(6)
    n = 3000
    pos = [rng.random(n), rng.random(n) * 0.05, rng.random(n) * 0.05]
    pos[0][:50] = 0.0
    pos[0][50:100] = np.nextafter(1.0, 0)
    vel = [rng.normal(0, 1, n) for _ in range(3)]
    vel[0][100:200] = vel[0][99]
    s = ki.Setup(n=n, box=(1.0, 0.05, 0.05), bc=(0, 0, 0), d0=0.01, dt=0.01, seed=7,
                 name="equilibrium_slab")
    for prec, kern in ((FP64, 0), (FP32, 0), (FP64, 2), (FP32, 2), (FP64, 1), (FP32, 3)):
        sim, st, oc, _ = run_both(s, 20, prec, arrays=pos + vel, search_kernel=kern)
        assert_same_counts(sim.counts(), oc)
        assert_same_state(sim, st)
    # reflecting box on all axes with a static upper wall
    s = ki.Setup(n=2000, box=(1.0, 0.5, 0.7), bc=(1, 1, 1), piston_x0=1.0, piston_u=0.0,
                 d0=0.02, dt=0.02, seed=8, name="walls")
    rng = np.random.default_rng(8)
    arrays = [rng.random(2000) * b for b in (1.0, 0.5, 0.7)] + [rng.normal(0, 2, 2000) for _ in range(3)]
    for prec in (FP64, FP32):
        sim, st, oc, _ = run_both(s, 30, prec, arrays=arrays)
        assert_same_counts(sim.counts(), oc)
        assert_same_state(sim, st)


def test_overflowing_pair_buffer_grows_and_results_are_unchanged():
    s = ki.equilibrium_setup(n=4096, seed=10)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    oc, _ = oracle.run(s, st, 0, 30)
    sim = gpu_sim(s, arrays, FP64, edge_cap=8)
    sim.step(30).sync()
    assert_same_counts(sim.counts(), oc)
    assert_same_state(sim, st)


def test_resume_from_observed_state_is_bit_exact():
    s = ki.piston_setup(n=6000, seed=11, box=(2.0, 0.5, 0.5), profile_bins=0, profile_every=0)
    arrays = ki.initial_state(s)
    full = gpu_sim(s, arrays, FP32).step(30).sync()
    half = gpu_sim(s, arrays, FP32).step(12).sync()
    mid, last = half.state()
    rest = gpu_sim(s, mid, FP32, last=last, step0=12).step(18).sync()
    a, la = full.state()
    b, lb = rest.state()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(la, lb)
    assert rest.step_index() == 30


def test_profiles_match_oracle_within_summation_bound():
    s = ki.piston_setup(n=1 << 14, seed=12, box=(8.0, 0.125, 0.125), profile_bins=256,
                        profile_every=50)
    sim, st, oc, oprof = run_both(s, 150)
    gprof = sim.profiles()
    assert gprof.shape == oprof.shape == (3, 256, 7)
    assert np.array_equal(gprof[:, :, 0], oprof[:, :, 0])  # counts are integers
    # the oracle sums in id order in binary64: |error| <= (n-1) u sum|terms|; the GPU
    # sum is exact to 2^-64 per term and rounded once
    u = 2.0 ** -53
    _, _ = sim.state()
    cnt = oprof[:, :, 0]
    for q in range(1, 7):
        mag_bound = np.abs(oprof[:, :, q]) + 1e-300
        # sum |terms| <= count * max|term|: bound with the per-bin second moments
        sq = oprof[:, :, 4 + (q - 1) % 3]
        abs_sum = np.sqrt(np.maximum(cnt * sq, 0)) if q <= 3 else sq
        tol = (cnt + 2) * u * abs_sum + cnt * 2.0 ** -64 + 2 * u * mag_bound
        assert np.all(np.abs(gprof[:, :, q] - oprof[:, :, q]) <= tol), q


def test_full_size_piston_tube_two_steps_bit_exact():
    """The 2^20-particle piston tube at full size: two steps against the oracle."""
    s = ki.piston_setup(n=1 << 20, seed=2)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    oc, _ = oracle.run(s, st, 0, 2)
    for prec in (FP64, FP32):
        sim = gpu_sim(s, arrays, prec).step(2).sync()
        assert_same_counts(sim.counts(), oc)
        assert_same_state(sim, st)


def test_group_of_uneven_runs_equals_each_run_alone():
    setups = ki.ensemble_setups(count=6, lo=1 << 10, hi=1 << 14, steps=25)
    arrays = [ki.initial_state(s) for s in setups]
    sims = [gpu_sim(s, a, FP32) for s, a in zip(setups, arrays)]
    g = kmc.Group(sims)
    budgets = [25, 10, 25, 17, 3, 25]
    for sim, b in zip(sims, budgets):
        g.budget(sim, b)
    g.step(25)
    g.sync()
    for sim, b in zip(sims, budgets):
        assert g.steps_left(sim) == 0
    for s, a, sim, b in zip(setups, arrays, sims, budgets):
        st = oracle.State(a)
        oc, _ = oracle.run(s, st, 0, b)
        assert_same_counts(sim.counts(), oc)
        assert_same_state(sim, st)
    g.close()


@pytest.mark.parametrize("stencil", [1, 2])
def test_row_search_periodic_x_wrap(stencil):
    """Short periodic x axis (few cells) with sparse cells: stencil rows of particles
    near either end wrap and are searched through the periodic image."""
    rng = np.random.default_rng(31)
    n = 3000
    box = (0.3, 1.0, 1.0)
    pos = [np.minimum(rng.random(n) * b, np.nextafter(b, 0)) for b in box]
    vel = [rng.normal(0, 1, n) for _ in range(3)]
    s = ki.Setup(n=n, box=box, bc=(0, 0, 0), d0=0.01, dt=0.01, seed=31, name="equilibrium_short")
    for prec in (FP32,):
        sim, st, oc, _ = run_both(s, 15, prec, arrays=pos + vel, search_kernel=3, stencil=stencil)
        assert_same_counts(sim.counts(), oc)
        assert_same_state(sim, st)


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("kernel,stencil", [(0, 1), (1, 1), (2, 1), (3, 1), (3, 2)])
def test_speed_split_forced_is_bit_exact(precision, kernel, stencil):
    """Fast particles in a second population (threshold cycling through all trial
    values step by step), searched by the fast-particle kernel: same trajectory."""
    s = ki.piston_setup(n=1 << 15, seed=41, box=(8.0, 0.25, 0.25), profile_bins=0,
                        profile_every=0)
    flags = kmc.KMC_FLAG_FORCE_SPLIT
    sim, st, oc, _ = run_both(s, 40, precision, search_kernel=kernel, stencil=stencil, flags=flags)
    assert_same_counts(sim.counts(), oc)
    assert_same_state(sim, st)


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_speed_split_forced_equilibrium_and_no_split(precision):
    s = ki.equilibrium_setup(n=8192, seed=42, L=1.3, dt=0.005)
    for flags in (kmc.KMC_FLAG_FORCE_SPLIT, kmc.KMC_FLAG_NO_SPLIT):
        sim, st, oc, _ = run_both(s, 30, precision, flags=flags)
        assert_same_counts(sim.counts(), oc)
        assert_same_state(sim, st)


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("kernel", [0, 3])
def test_spherical_blast_downscale_bit_exact(precision, kernel):
    """Hot dense sphere (8x density, 100x temperature) in a periodic cube, the same
    geometry and background mean free path at 2^16 particles: the fast tail drives the
    speed split every step.  Trajectory and counts equal the oracle's."""
    s = ki.blast_setup(n=1 << 16, seed=3, lam_bg=0.005, steps=25)
    sim, st, oc, _ = run_both(s, 25, precision, search_kernel=kernel)
    assert_same_counts(sim.counts(), oc)
    assert_same_state(sim, st)
    assert sum(c["collisions"] for c in oc) > 1000


@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_long_periodic_box_near_thresholds_binary32_equals_binary64(kernel):
    """Box coordinates up to 48 (the binary32 mirror's largest rounding errors) with
    positions and velocities on coarse lattices, so that many pairs sit on or within
    ulps of the t* = 0, t* = dt and d_min = d0 thresholds, some across the periodic
    boundary: both precisions give the oracle's candidate list."""
    rng = np.random.default_rng(77)
    n = 6000
    box = (48.0, 0.75, 0.75)
    pos = [np.minimum(np.round(rng.random(n) * b * 64) / 64, np.nextafter(b, 0)) for b in box]
    pos[0][:300] = np.nextafter(box[0], 0) - np.round(rng.random(300) * 8) / 64
    vel = [np.round(rng.normal(0, 1, n) * 8) / 8 for _ in range(3)]
    s = ki.Setup(n=n, box=box, bc=(0, 0, 0), d0=1 / 32, dt=1 / 16, seed=77,
                 name="equilibrium_long_lattice")
    st = oracle.State(pos + vel)
    pi, pj, _, _ = oracle.candidate_pairs(s, st)
    assert len(pi) > 200
    for prec in (FP64, FP32):
        sim = gpu_sim(s, pos + vel, prec, search_kernel=kernel).step(1).sync()
        assert np.array_equal(sim.edges(), np.stack([pi, pj], axis=1))


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_planar_equal_speed_reflecting_square_bit_exact(precision, kernel):
    """The paper's 2D runs: equal speeds in random in-plane directions, reflecting
    walls, a z extent of one cell (9-cell stencil), isotropic in-plane scatter."""
    s = ki.equal_speed_setup(n=8192, seed=12, d0=0.002, dt=0.005, steps=120)
    sim, st, oc, _ = run_both(s, 120, precision, search_kernel=kernel)
    assert_same_counts(sim.counts(), oc)
    assert_same_state(sim, st)
    assert sum(c["collisions"] for c in oc) > 20000
    arrays, _ = sim.state()
    assert np.all(arrays[5] == 0.0)


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_planar_periodic_square_pair_lists_and_forced_split(precision):
    s = ki.equal_speed_setup(n=6000, seed=13, d0=0.004, dt=0.01)
    s = s.with_(bc=(ki.PERIODIC, ki.PERIODIC, ki.REFLECT))
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    sim = gpu_sim(s, arrays, precision=precision, flags=kmc.KMC_FLAG_FORCE_SPLIT)
    for step in range(8):
        pi, pj, _, _ = oracle.candidate_pairs(s, st)
        counts, partner, _ = oracle.step(s, st, step)
        sim.step(1).sync()
        e = sim.edges()
        assert np.array_equal(e, np.stack([pi, pj], axis=1)), f"step {step}"
        assert np.array_equal(sim.partners(), partner), f"step {step}"
    assert_same_state(sim, st)


def test_planar_rejects_out_of_plane_velocity():
    s = ki.equal_speed_setup(n=512, seed=14)
    arrays = ki.initial_state(s)
    arrays[5] = arrays[5].copy()
    arrays[5][77] = 1e-300
    with pytest.raises(kmc.KmcError) as e:
        gpu_sim(s, arrays)
    assert e.value.code == kmc.KMC_EINVAL and "vz" in str(e.value)


def _absorbing_setup(n=6000, seed=71, bc=(ki.ABSORB, ki.REFLECT, ki.PERIODIC), dt=0.01):
    s = ki.equilibrium_setup(n=n, seed=seed, d0=0.02, dt=dt)
    return s.with_(bc=bc, piston_x0=1.0, piston_u=0.0)


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_absorbing_walls_bit_exact(precision, kernel):
    """Absorptive walls (Sec. 2): the particles that leave are the oracle's, step by
    step, and keep the oracle's exit positions and velocities."""
    s = _absorbing_setup()
    sim, st, oc, _ = run_both(s, 60, precision, search_kernel=kernel)
    assert_same_counts(sim.counts(), oc)
    assert_same_state(sim, st)
    assert oc[-1]["live"] < 0.8 * s.n
    assert int((st.last == oracle.ABSORBED).sum()) == s.n - oc[-1]["live"]


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_absorbing_pair_lists_forced_split_and_resume(precision):
    s = _absorbing_setup(n=8000, seed=72, bc=(ki.ABSORB, ki.ABSORB, ki.ABSORB))
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    sim = gpu_sim(s, arrays, precision=precision, flags=kmc.KMC_FLAG_FORCE_SPLIT)
    for step in range(10):
        pi, pj, _, _ = oracle.candidate_pairs(s, st)
        counts, partner, _ = oracle.step(s, st, step)
        sim.step(1).sync()
        assert np.array_equal(sim.edges(), np.stack([pi, pj], axis=1)), f"step {step}"
        assert np.array_equal(sim.partners(), partner), f"step {step}"
    assert_same_state(sim, st)
    # resume from the observed state (absorbed particles flagged in last)
    mid, last = sim.state()
    assert np.any(last == kmc.KMC_ABSORBED)
    rest = gpu_sim(s, mid, precision, last=last, step0=10, flags=kmc.KMC_FLAG_FORCE_SPLIT)
    rest.step(15).sync()
    oc, _ = oracle.run(s, st, 10, 15)
    assert_same_counts(rest.counts(), oc)
    assert_same_state(rest, st)


def test_absorbing_box_empties_and_groups_mix():
    """Every particle leaves (live reaches 0, the steps after that are empty), and a
    group mixing absorbing and periodic runs equals each run alone."""
    s = _absorbing_setup(n=3000, seed=73, bc=(ki.ABSORB,) * 3, dt=0.05)
    sim, st, oc, _ = run_both(s, 130, FP32)  # the last particle leaves at step 106
    assert_same_counts(sim.counts(), oc)
    assert_same_state(sim, st)
    assert oc[-1]["live"] == 0 and np.all(st.last == oracle.ABSORBED)
    setups = [_absorbing_setup(n=2000 + 500 * k, seed=80 + k,
                               bc=(ki.ABSORB, ki.PERIODIC, ki.PERIODIC) if k % 2 else (ki.PERIODIC,) * 3)
              for k in range(4)]
    arrays = [ki.initial_state(q) for q in setups]
    sims = [gpu_sim(q, a, FP32) for q, a in zip(setups, arrays)]
    g = kmc.Group(sims)
    for x in sims:
        g.budget(x, 30)
    g.step(30)
    g.sync()
    for q, a, x in zip(setups, arrays, sims):
        st = oracle.State(a)
        oc, _ = oracle.run(q, st, 0, 30)
        assert_same_counts(x.counts(), oc)
        assert_same_state(x, st)
    g.close()


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_mixture_bit_exact(precision, kernel):
    """Binary mixture (Sec. 2: per-particle mass and effective radius): contact at
    r_i + r_j, mass-weighted scatter, bit-identical to the oracle."""
    s = ki.mixture_setup(n=6000, seed=91, mass_b=4.0, kT_b=2.0)
    sim, st, oc, _ = run_both(s, 60, precision, search_kernel=kernel)
    assert_same_counts(sim.counts(), oc)
    assert_same_state(sim, st)
    assert sum(c["collisions"] for c in oc) > 5000


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_mixture_pair_lists_split_and_absorbing_walls(precision):
    s = ki.mixture_setup(n=8000, seed=92, mass_b=9.0, d_a=0.01, d_b=0.03)
    s = s.with_(bc=(ki.ABSORB, ki.PERIODIC, ki.REFLECT), piston_x0=1.0, piston_u=0.0)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    sim = gpu_sim(s, arrays, precision=precision, flags=kmc.KMC_FLAG_FORCE_SPLIT)
    for step in range(12):
        pi, pj, _, _ = oracle.candidate_pairs(s, st)
        counts, partner, _ = oracle.step(s, st, step)
        sim.step(1).sync()
        assert np.array_equal(sim.edges(), np.stack([pi, pj], axis=1)), f"step {step}"
        assert np.array_equal(sim.partners(), partner), f"step {step}"
    assert_same_state(sim, st)


def test_mixture_rejects_bad_species_index():
    s = ki.mixture_setup(n=1000, seed=93)
    arrays = ki.initial_state(s)
    sp = s.species.copy()
    sp[500] = 2  # two species: 0 and 1
    with pytest.raises(kmc.KmcError) as e:
        kmc.Simulation(kmc.params_from_setup(s), arrays, mixture=(sp, s.masses, s.radii))
    assert e.value.code == kmc.KMC_EINVAL and "species" in str(e.value)


def test_group_mixing_every_variant_equals_each_alone():
    """One group holding a plain gas, a mixture, an absorbing box, a planar gas and a
    planar absorbing mixture: the plan launches the general forms of the kernels,
    which must leave each member's results those of the oracle."""
    plain = ki.equilibrium_setup(n=3000, seed=95)
    mix = ki.mixture_setup(n=3500, seed=96, mass_b=3.0)
    absorb = _absorbing_setup(n=2500, seed=97, bc=(ki.ABSORB, ki.REFLECT, ki.PERIODIC))
    planar = ki.equal_speed_setup(n=4000, seed=98, d0=0.004, dt=0.01)
    pmix = ki.equal_speed_setup(n=3000, seed=99, d0=0.006, dt=0.01)
    n = pmix.n
    pmix = pmix.with_(bc=(ki.ABSORB, ki.PERIODIC, ki.REFLECT), piston_x0=1.0,
                      species=(np.arange(n) % 3).astype(np.uint8), masses=(1.0, 2.5, 0.5),
                      radii=(0.003, 0.002, 0.001))
    setups = [plain, mix, absorb, planar, pmix]
    arrays = [ki.initial_state(q) for q in setups]
    for prec in (FP64, FP32):
        sims = [gpu_sim(q, a, prec) for q, a in zip(setups, arrays)]
        g = kmc.Group(sims)
        for x in sims:
            g.budget(x, 25)
        g.step(25)
        g.sync()
        for q, a, x in zip(setups, arrays, sims):
            st = oracle.State(a)
            oc, _ = oracle.run(q, st, 0, 25)
            assert_same_counts(x.counts(), oc)
            assert_same_state(x, st)
            assert sum(c["collisions"] for c in oc) > 0
        g.close()


def test_group_of_more_members_than_a_block_has_threads_is_exact():
    """The matching kernels read the members' item counts a block's width (256) at a
    time and carry the dealing position from one chunk of members to the next; a group
    of 300 small runs (boxes and tubes of uneven size) crosses that boundary.  Every
    member ends where the oracle says."""
    setups = []
    for k in range(300):
        if k % 2 == 0:
            setups.append(ki.equilibrium_setup(n=300 + (k * 37) % 500, seed=2000 + k))
        else:
            setups.append(ki.piston_setup(n=2000 + (k * 37) % 2000, seed=2000 + k,
                                          profile_bins=0, profile_every=0))
    arrays = [ki.initial_state(q) for q in setups]
    sims = [gpu_sim(q, a, FP32) for q, a in zip(setups, arrays)]
    g = kmc.Group(sims)
    for x in sims:
        g.budget(x, 4)
    g.step(4)
    g.sync()
    for q, a, x in zip(setups, arrays, sims):
        assert g.steps_left(x) == 0
        st = oracle.State(a)
        oc, _ = oracle.run(q, st, 0, 4)
        assert_same_counts(x.counts(), oc)
        assert_same_state(x, st)
    g.close()


@pytest.mark.parametrize("search", [kmc.KMC_SEARCH_CELL, kmc.KMC_SEARCH_ROW])
def test_group_members_overflowing_mid_search_leave_the_others_exact(search):
    """Batch kernels deal the members' cells and pairs to the grid as one sequence.  A
    member whose pair buffer fills sets its status while the search runs; blocks that
    look at it earlier or later must still agree on where every other member's work
    falls, so no cell of another member is searched twice or missed.  Members 0 and 3
    overflow in every step here; all six end where the oracle says."""
    setups = [ki.equilibrium_setup(n=2000 + 500 * k, seed=140 + k) for k in range(6)]
    arrays = [ki.initial_state(q) for q in setups]
    sims = [gpu_sim(q, a, FP32, edge_cap=(8 if k in (0, 3) else 0), search_kernel=search)
            for k, (q, a) in enumerate(zip(setups, arrays))]
    g = kmc.Group(sims)
    for x in sims:
        g.budget(x, 6)
    g.step(6)
    g.sync()
    for q, a, x in zip(setups, arrays, sims):
        assert g.steps_left(x) == 0
        st = oracle.State(a)
        oc, _ = oracle.run(q, st, 0, 6)
        assert_same_counts(x.counts(), oc)
        assert_same_state(x, st)
    g.close()


def test_group_member_whose_pair_buffer_overflows_catches_up_at_sync():
    """A member whose candidate-pair buffer overflows in a group step is skipped by the
    group's later steps; the group's sync grows its buffer and runs the steps it
    missed, so after the sync every member is where its budget says."""
    setups = [ki.equilibrium_setup(n=3000 + 700 * k, seed=110 + k) for k in range(3)]
    arrays = [ki.initial_state(q) for q in setups]
    sims = [gpu_sim(q, a, FP32, edge_cap=(8 if k == 1 else 0))
            for k, (q, a) in enumerate(zip(setups, arrays))]
    g = kmc.Group(sims)
    budgets = [30, 30, 12]
    for x, b in zip(sims, budgets):
        g.budget(x, b)
    g.step(10)
    g.sync()
    g.step(20)
    g.sync()
    for q, a, x, b in zip(setups, arrays, sims, budgets):
        assert g.steps_left(x) == 0
        st = oracle.State(a)
        oc, _ = oracle.run(q, st, 0, b)
        assert_same_counts(x.counts(), oc)
        assert_same_state(x, st)
    g.close()
