"""Pins of the oracle's matching, collision update and boundaries against brute
force, conservation laws and closed-form kinetic theory (no GPU needed).

* Mutual choice (Sec. 2): a brute-force rendering of the rounds on tiny systems,
  plus invariants (disjoint pairs, mutual best within the round, no mutual best
  left unmatched).
* Collision update: momentum and energy of every colliding pair conserved within
  the rounding bound of the update.
* Hard-sphere collision rate (1/2) n^2 sigma <|g|> with <|g|> = sqrt(16 kT / (pi m)).
* Piston shock: Rankine-Hugoniot jump conditions of an ideal monatomic gas.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import kmc_inputs as ki
import oracle

NONE = oracle.NONE
U = 2.0 ** -53


def _brute_matching(n, pairs, keys, max_rounds):
    """Mutual choice written from the definition: each round, each unmatched particle
    points at its unmatched candidate of least (d2, t, id); mutual pointers collide."""
    cand = {i: [] for i in range(n)}
    for (i, j), (d2, t) in zip(pairs, keys):
        cand[i].append((d2, t, j))
        cand[j].append((d2, t, i))
    partner = [NONE] * n
    rounds = []
    for _ in range(max_rounds):
        best = {}
        for i in range(n):
            if partner[i] != NONE:
                continue
            opts = [c for c in cand[i] if partner[c[2]] == NONE]
            if opts:
                best[i] = min(opts)[2]
        newly = [(i, j) for i, j in best.items() if i < j and best.get(j) == i]
        for i, j in newly:
            partner[i], partner[j] = j, i
        rounds.append(len(newly))
        if not newly:
            break
    return partner, rounds


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_matching_brute_force_tiny(seed):
    # dense, slow-moving gas so that most particles have several candidates
    n = 60
    s = ki.Setup(n=n, box=(1.0, 1.0, 1.0), bc=(0, 0, 0), d0=0.25, dt=0.2, seed=seed,
                 name="equilibrium_tiny")
    st = oracle.State(ki.equilibrium_state(n, seed))
    pi, pj, d2, t = oracle.candidate_pairs(s, st, search=0)
    assert len(pi) > n  # several candidates per particle
    want, rounds = _brute_matching(n, list(zip(pi.tolist(), pj.tolist())),
                                   list(zip(d2.tolist(), t.tolist())), s.max_rounds)
    st2 = st.copy()
    counts, partner, _ = oracle.step(s, st2, 0, search=0)
    assert partner.tolist() == want
    assert counts["round_pairs"][: len(rounds)] == rounds
    assert counts["collisions"] == sum(rounds)
    assert counts["edges"] == len(pi)
    # invariants
    p = partner.tolist()
    for i, j in enumerate(p):
        if j != NONE:
            assert p[j] == i and j != i


def _pair_bounds_check(before, after, partner):
    """Exact (rational) momentum and energy change of each colliding pair."""
    worst_p = 0.0
    worst_e = 0.0
    n = len(partner)
    for a in range(n):
        b = int(partner[a])
        if b == NONE or b < a:
            continue
        va = [before[3 + k][a] for k in range(3)]
        vb = [before[3 + k][b] for k in range(3)]
        wa = [after[3 + k][a] for k in range(3)]
        wb = [after[3 + k][b] for k in range(3)]
        vmax = max(math.sqrt(sum(x * x for x in va)), math.sqrt(sum(x * x for x in vb)))
        for k in range(3):
            dp = (Fraction(wa[k]) + Fraction(wb[k])) - (Fraction(va[k]) + Fraction(vb[k]))
            # fl(va+vb)*0.5 then fl(V+p) + fl(V-p): at most 3 roundings, each <= u*2vmax
            assert abs(float(dp)) <= 6 * U * vmax
            worst_p = max(worst_p, abs(float(dp)) / (U * vmax))
        e0 = sum(Fraction(x) ** 2 for x in va + vb)
        e1 = sum(Fraction(x) ** 2 for x in wa + wb)
        # relative bound from rounding in V, G, n-hat and V +- p (first order, 16 u)
        assert abs(float(e1 - e0)) <= 16 * U * float(e0)
        worst_e = max(worst_e, abs(float(e1 - e0)) / (U * float(e0)))
    return worst_p, worst_e


def test_conservation_per_collision():
    s = ki.equilibrium_setup(n=4096, seed=5)
    st = oracle.State(ki.initial_state(s))
    total = 0
    for step in range(5):
        before = [x.copy() for x in st.a]
        counts, partner, _ = oracle.step(s, st, step)
        total += counts["collisions"]
        _pair_bounds_check(before, st.a, partner)
        # velocities of non-colliders untouched (periodic box: no wall)
        idle = partner == NONE
        for k in range(3, 6):
            assert np.array_equal(before[k][idle], st.a[k][idle])
    assert total > 500


def _sample_kT(state):
    v = np.stack(state.a[3:6], axis=1)
    n = v.shape[0]
    return float(((v - v.mean(axis=0)) ** 2).sum() / (3 * (n - 1)))


def test_collision_rate_step0_closed_form():
    """Expected candidate pairs at step 0: C(N,2) * pi d0^2 <|g|> dt / V with
    <|g|> = sqrt(16 kT/(pi m)), summed over independent seeds, within 3 sigma."""
    got = 0
    expect = 0.0
    for seed in range(100, 140):
        s = ki.equilibrium_setup(n=4096, seed=seed)
        st = oracle.State(ki.initial_state(s))
        pi, _, _, _ = oracle.candidate_pairs(s, st)
        got += len(pi)
        kT = _sample_kT(st)
        g = math.sqrt(16 * kT / math.pi)
        expect += s.n * (s.n - 1) / 2 * math.pi * s.d0 ** 2 * g * s.dt / 1.0
    sigma = math.sqrt(expect)
    assert abs(got - expect) < 3 * sigma, (got, expect, sigma)


def test_collision_rate_200_steps():
    """Matched collisions over 200 steps vs (1/2) n^2 sigma <|g|> V dt per step, at
    dt = 0.001 where one-collision-per-step truncation costs only ~mu/2 = 0.6%."""
    s = ki.equilibrium_setup(n=4096, seed=1, dt=0.001)
    st = oracle.State(ki.initial_state(s))
    kT = _sample_kT(st)
    counts, _ = oracle.run(s, st, 0, 200)
    coll = sum(c["collisions"] for c in counts)
    g = math.sqrt(16 * kT / math.pi)
    expect = 0.5 * s.n ** 2 * math.pi * s.d0 ** 2 * g * s.dt * 200
    assert abs(coll - expect) < 3 * math.sqrt(expect), (coll, expect)
    # temperature is conserved in the periodic box (elastic collisions only)
    assert abs(_sample_kT(st) - kT) < 1e-9 * kT


def test_resume_is_bit_exact():
    s = ki.piston_setup(n=3000, seed=8, box=(2.0, 0.5, 0.5), profile_bins=0, profile_every=0)
    a = oracle.State(ki.initial_state(s))
    b = a.copy()
    ca, _ = oracle.run(s, a, 0, 12)
    cb1, _ = oracle.run(s, b, 0, 5)
    c = oracle.State(b.a, b.last)  # checkpoint / restore
    cb2, _ = oracle.run(s, c, 5, 7)
    assert ca == cb1 + cb2
    for x, y in zip(a.a, c.a):
        assert np.array_equal(x, y)
    assert np.array_equal(a.last, c.last)


def test_walls_and_piston_keep_particles_inside():
    s = ki.piston_setup(n=5000, seed=9, box=(2.0, 0.5, 0.5), u_p=2.0, profile_bins=0,
                        profile_every=0)
    st = oracle.State(ki.initial_state(s))
    e0 = float(sum((v ** 2).sum() for v in st.a[3:6]))
    steps = 150
    oracle.run(s, st, 0, steps)
    X = s.piston_x0 - s.piston_u * (steps * s.dt)
    x = st.a[0]
    assert x.min() >= 0.0 and x.max() <= X
    for k in (1, 2):
        assert st.a[k].min() >= 0.0 and st.a[k].max() < s.box[k]
    # the piston does work on the gas
    assert float(sum((v ** 2).sum() for v in st.a[3:6])) > e0


def test_piston_reflection_is_specular_in_wall_frame():
    # one particle, no partner: it hits the piston and must leave with -v - 2u
    s = ki.Setup(n=1, box=(1.0, 1.0, 1.0), bc=(1, 0, 0), piston_x0=1.0, piston_u=0.5,
                 d0=0.01, dt=0.1, name="piston_single")
    st = oracle.State([np.array([0.95]), np.array([0.5]), np.array([0.5]),
                       np.array([1.0]), np.array([0.0]), np.array([0.0])])
    oracle.step(s, st, 0)
    X = 1.0 - 0.5 * 0.1
    assert st.a[3][0] == -1.0 - 1.0
    assert st.a[0][0] == (X + X) - (0.95 + 1.0 * 0.1)


@pytest.mark.slow
def test_rankine_hugoniot_piston_shock():
    """Piston driven shock in an ideal monatomic gas (gamma = 5/3):
    u_s = (g+1) u_p/4 + sqrt(((g+1) u_p/4)^2 + c0^2), rho1/rho0 = u_s/(u_s - u_p),
    kT1 = (kT0 + u_s u_p) rho0/rho1.  Each within 2%."""
    n = 1 << 16
    box = (8.0, 0.25, 0.25)
    s = ki.piston_setup(n=n, seed=2, box=box, u_p=2.0, steps=1000, profile_bins=256,
                        profile_every=100)
    st = oracle.State(ki.initial_state(s))
    kT0 = float(np.mean([np.var(v) for v in st.a[3:6]]))
    counts, prof = oracle.run(s, st, 0, s.steps)
    gam = 5.0 / 3.0
    up = s.piston_u
    c0 = math.sqrt(gam * kT0)
    a = (gam + 1) * up / 4
    us = a + math.sqrt(a * a + c0 * c0)
    ratio = us / (us - up)
    kT1 = (kT0 + us * up) / ratio
    width = box[0] / 256
    area = box[1] * box[2]
    n0 = n / (box[0] * area)
    times = [(k + 1) * 100 * s.dt for k in range(prof.shape[0])]
    centers = (np.arange(256) + 0.5) * width
    lam1 = 0.02 / ratio
    shock_pos = []
    plateau_n, plateau_T, plateau_u = [], [], []
    for snap, t in zip(prof, times):
        cnt = snap[:, 0]
        dens = cnt / (width * area)
        piston = s.piston_x0 - up * t
        # plateau estimate from bins well behind the shock front
        sel = (centers < piston - 5 * lam1) & (centers > piston - 0.5 * (us - up) * t)
        n1 = dens[sel].mean()
        half = 0.5 * (n0 + n1)
        # shock position: first upward crossing of the half level, scanning from the
        # undisturbed gas (linear interpolation between bin centres)
        k = int(np.argmax(dens > half))
        f = (half - dens[k - 1]) / (dens[k] - dens[k - 1])
        xs = centers[k - 1] + f * width
        shock_pos.append(xs)
        if t >= 0.5:
            pl = (centers > xs + 5 * lam1) & (centers < piston - 5 * lam1)
            c = cnt[pl]
            mv = snap[pl, 1:4] / c[:, None]
            var = snap[pl, 4:7] / c[:, None] - mv ** 2
            plateau_n.append(cnt[pl].sum() / (pl.sum() * width * area))
            plateau_T.append(float((var.mean(axis=1) * c).sum() / c.sum()))
            plateau_u.append(float(snap[pl, 1].sum() / c.sum()))
    t_arr = np.array(times)
    m = t_arr >= 0.5
    slope = np.polyfit(t_arr[m], np.array(shock_pos)[m], 1)[0]
    us_meas = -slope
    assert abs(us_meas / us - 1) < 0.02, (us_meas, us)
    assert abs(np.mean(plateau_n) / n0 / ratio - 1) < 0.02, (np.mean(plateau_n) / n0, ratio)
    assert abs(np.mean(plateau_T) / kT1 - 1) < 0.02, (np.mean(plateau_T), kT1)
    assert abs(np.mean(plateau_u) / (-up) - 1) < 0.02
