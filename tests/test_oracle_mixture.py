"""Pins of the oracle's mixtures (Sec. 2: every particle carries a mass and an
effective radius; a pair is in contact at r_i + r_j).

Checked against facts fixed outside the oracle: geometry of single pairs (contact at
r_i + r_j, not at the search reach d0); a mixture of identical species whose mass is
a power of two is the plain gas, bit for bit (the update reduces exactly); per-collision momentum sum(m v) and
energy sum(m v^2) within rounding; the step-0 candidate count of a Maxwellian
mixture, sum over species pairs of N_ab pi (r_a + r_b)^2 <|g_ab|> dt / V with
<|g_ab|> = sqrt(8/pi (kT_a/m_a + kT_b/m_b)); the cell search equals brute force; two
species at different temperatures relax to one temperature (equipartition).
"""
import math
from dataclasses import replace
from fractions import Fraction

import numpy as np
import pytest

import kmc_inputs as ki
import oracle

U = 2.0 ** -53
NONE = 0xFFFFFFFF


def _pair(sp, radii, masses, b, d0=0.032):
    """Two particles, species sp[0], sp[1], approaching head-on along x with impact
    parameter b along y."""
    s = ki.Setup(n=2, box=(1.0, 1.0, 1.0), bc=(0, 0, 0), d0=d0, dt=0.1, seed=3,
                 name="mixture_pair", species=np.array(sp, np.uint8), masses=masses,
                 radii=radii)
    arrays = [np.array([0.40, 0.45]), np.array([0.5, 0.5 + b]), np.array([0.5, 0.5]),
              np.array([0.3, -0.3]), np.zeros(2), np.zeros(2)]
    return s, oracle.State(arrays)


def test_contact_distance_is_the_sum_of_radii():
    radii, masses = (0.008, 0.016), (1.0, 4.0)
    for sp, contact in (((0, 0), 0.016), ((0, 1), 0.024), ((1, 0), 0.024), ((1, 1), 0.032)):
        for f, want in ((0.95, True), (1.05, False)):
            s, st = _pair(sp, radii, masses, f * contact)
            ok, d2, t = oracle.pair(s, st, 0, 1)
            assert ok == want, (sp, f)
            if ok:
                assert abs(math.sqrt(d2) - f * contact) < 1e-12


def test_identical_species_reproduce_the_plain_gas_bit_for_bit():
    plain = ki.equilibrium_setup(n=4096, seed=9)
    arrays = ki.initial_state(plain)
    ref = oracle.State(arrays)
    rc, _ = oracle.run(plain, ref, 0, 30)
    # equal masses that are powers of two: every mass product and the division by M
    # are exact scalings, so the update is the plain one bit for bit
    for masses in ((1.0,), (2.0, 2.0), (0.25, 0.25, 0.25)):
        k = len(masses)
        mix = replace(plain, species=(np.arange(plain.n) % k).astype(np.uint8), masses=masses,
                      radii=(0.5 * plain.d0,) * k)
        st = oracle.State(arrays)
        mc, _ = oracle.run(mix, st, 0, 30)
        assert [c["collisions"] for c in mc] == [c["collisions"] for c in rc]
        for a, b in zip(st.a, ref.a):
            assert np.array_equal(a, b)
        assert np.array_equal(st.last, ref.last)


def test_mixture_collisions_conserve_mass_weighted_momentum_and_energy():
    s = ki.mixture_setup(n=5000, seed=11, mass_b=7.0)
    m = np.asarray(s.masses)[s.species]
    st = oracle.State(ki.initial_state(s))
    total = 0
    for step in range(4):
        before = [x.copy() for x in st.a]
        counts, partner, _ = oracle.step(s, st, step)
        total += counts["collisions"]
        for a in range(s.n):
            b = int(partner[a])
            if b == NONE or b < a:
                continue
            ma, mb = Fraction(m[a]), Fraction(m[b])
            va = [Fraction(before[3 + k][a]) for k in range(3)]
            vb = [Fraction(before[3 + k][b]) for k in range(3)]
            wa = [Fraction(st.a[3 + k][a]) for k in range(3)]
            wb = [Fraction(st.a[3 + k][b]) for k in range(3)]
            pmax = float(max(ma, mb)) * max(math.sqrt(sum(float(x) ** 2 for x in va)),
                                            math.sqrt(sum(float(x) ** 2 for x in vb)))
            for k in range(3):
                dp = (ma * wa[k] + mb * wb[k]) - (ma * va[k] + mb * vb[k])
                assert abs(float(dp)) <= 16 * U * pmax
            e0 = sum(ma * x * x for x in va) + sum(mb * x * x for x in vb)
            e1 = sum(ma * x * x for x in wa) + sum(mb * x * x for x in wb)
            assert abs(float(e1 - e0)) <= 32 * U * float(e0)
    assert total > 300


def test_mixture_candidate_rate_step0_closed_form():
    got = 0
    expect = 0.0
    for seed in range(500, 530):
        s = ki.mixture_setup(n=4000, seed=seed, mass_b=4.0, kT_b=2.0)
        st = oracle.State(ki.initial_state(s))
        pi, pj, _, _ = oracle.candidate_pairs(s, st)
        got += len(pi)
        nb = int((s.species == 1).sum())
        counts = {(0, 0): (s.n - nb) * (s.n - nb - 1) / 2, (0, 1): (s.n - nb) * nb,
                  (1, 1): nb * (nb - 1) / 2}
        kT = s.extra["kT"]
        for (a, b), npair in counts.items():
            c = s.radii[a] + s.radii[b]
            g = math.sqrt(8.0 / math.pi * (kT[a] / s.masses[a] + kT[b] / s.masses[b]))
            expect += npair * math.pi * c * c * g * s.dt
    sigma = math.sqrt(expect)
    assert abs(got - expect) < 3 * sigma, (got, expect, sigma)


def test_mixture_cell_search_equals_brute_force():
    s = ki.mixture_setup(n=3000, seed=12)
    st = oracle.State(ki.initial_state(s))
    for _ in range(2):
        a = oracle.candidate_pairs(s, st, search=0)
        b = oracle.candidate_pairs(s, st, search=1)
        assert len(a[0]) > 0
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        oracle.run(s, st, 0, 5)


def test_two_temperatures_relax_to_one():
    """Species at kT 1 and 3 exchange energy until both carry the common temperature
    (equipartition: <m v^2>/3 per species equal)."""
    s = ki.mixture_setup(n=4000, seed=13, mass_b=3.0, kT_b=3.0, d_a=0.03, d_b=0.045,
                         dt=0.004)
    st = oracle.State(ki.initial_state(s))
    m = np.asarray(s.masses)[s.species]

    def temps():
        e = m * (st.a[3] ** 2 + st.a[4] ** 2 + st.a[5] ** 2) / 3.0
        return float(e[s.species == 0].mean()), float(e[s.species == 1].mean())

    t0 = temps()
    assert t0[1] > 2.5 * t0[0]
    counts, _ = oracle.run(s, st, 0, 150)
    assert sum(c["collisions"] for c in counts) > 6 * s.n
    ta, tb = temps()
    assert abs(ta - tb) < 0.05 * (ta + tb) / 2, (ta, tb)
