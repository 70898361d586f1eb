"""Pins of the oracle's absorbing walls (Sec. 2 lists absorptive walls beside
reflective and periodic ones).

Checked against facts fixed outside the oracle: without collisions a uniform slab
with absorbing faces keeps the fraction E[max(0, 1 - |v| t / L)] of its particles at
time t (free flight from a uniform start, v ~ N(0, 1)); absorbed particles keep the
position where they left and their velocity, so the total energy of all particles
is conserved; no absorbed particle is ever a candidate; the cell search still
equals brute force; counts add up.
"""
import math

import numpy as np
import pytest

import kmc_inputs as ki
import oracle


def _free_survival(a):
    # E[(1 - a|v|)_+], v ~ N(0, 1): erf(1/(a sqrt 2)) - 2a (1 - exp(-1/(2a^2))) / sqrt(2 pi)
    return math.erf(1.0 / (a * math.sqrt(2.0))) - 2.0 * a * (1.0 - math.exp(-0.5 / a ** 2)) / \
        math.sqrt(2.0 * math.pi)


@pytest.mark.parametrize("axis", [0, 2])
def test_free_flight_survival_closed_form(axis):
    # a thin slab along the absorbing axis keeps the cell search cheap
    n = 60000
    bc = [ki.PERIODIC] * 3
    bc[axis] = ki.ABSORB
    box = [4.0, 4.0, 4.0]
    box[axis] = 1.0
    s = ki.equilibrium_setup(n=n, seed=61, d0=1e-9, dt=0.02).with_(bc=tuple(bc), box=tuple(box))
    unit = ki.equilibrium_state(n, 61, 1.0)
    st = oracle.State([unit[k] * box[k] for k in range(3)] + unit[3:])
    counts, _ = oracle.run(s, st, 0, 20)
    assert sum(c["collisions"] for c in counts) == 0
    for k in (3, 6, 12, 20):
        live = counts[k - 1]["live"]
        p = _free_survival(k * s.dt / s.box[axis])
        sigma = math.sqrt(n * p * (1 - p))
        assert abs(live - n * p) < 4 * sigma, (k, live, n * p, sigma)


def _absorbing_gas(seed=62, n=6000):
    s = ki.equilibrium_setup(n=n, seed=seed, d0=0.02, dt=0.01)
    return s.with_(bc=(ki.ABSORB, ki.REFLECT, ki.PERIODIC), piston_x0=1.0, piston_u=0.0)


def test_absorbed_particles_leave_the_gas_for_good():
    s = _absorbing_gas()
    st = oracle.State(ki.initial_state(s))
    e0 = sum(float((x * x).sum()) for x in st.a[3:6])
    gone_before = np.zeros(s.n, bool)
    kept = None
    total_abs = 0
    for step in range(30):
        counts, partner, _ = oracle.step(s, st, step)
        gone = st.last == oracle.ABSORBED
        total_abs += counts["absorbed"]
        assert counts["absorbed"] == int(gone.sum() - gone_before.sum())
        assert counts["live"] == s.n - int(gone.sum())
        # absorbed this step: beyond an x face; absorbed earlier: frozen
        new = gone & ~gone_before
        x = st.a[0][new]
        assert np.all((x < 0.0) | (x > s.box[0]))
        if kept is not None:
            for k in range(6):
                assert np.array_equal(st.a[k][gone_before], kept[k])
        assert np.all(partner[gone_before] == oracle.NONE)
        kept = [a[gone].copy() for a in st.a]
        gone_before = gone
        # live particles are inside the box
        live = ~gone
        for k in range(3):
            assert np.all((st.a[k][live] >= 0.0) & (st.a[k][live] <= s.box[k]))
    assert total_abs > 300
    # elastic collisions conserve energy, absorption only removes particles
    e1 = sum(float((x * x).sum()) for x in st.a[3:6])
    assert abs(e1 - e0) < 1e-10 * e0
    # no candidate involves an absorbed particle; cell search = brute force
    a = oracle.candidate_pairs(s, st, search=0)
    b = oracle.candidate_pairs(s, st, search=1)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert len(a[0]) > 0
    gone = st.last == oracle.ABSORBED
    assert not np.any(gone[a[0]]) and not np.any(gone[a[1]])


def test_absorbed_particles_are_not_profiled():
    s = _absorbing_gas(seed=63).with_(profile_bins=16, profile_every=1, profile_range=1.0,
                                      bc=(ki.PERIODIC, ki.ABSORB, ki.PERIODIC))
    st = oracle.State(ki.initial_state(s))
    counts, prof = oracle.run(s, st, 0, 20)
    gone = int((st.last == oracle.ABSORBED).sum())
    assert gone > 100
    # absorbed through the y faces, with x still inside [0, 1): the last profile's
    # particle count equals the live count only if they are skipped
    assert int(round(prof[-1][:, 0].sum())) == counts[-1]["live"] == s.n - gone
