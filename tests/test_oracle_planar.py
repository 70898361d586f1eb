"""Pins of the oracle's planar (two-dimensional) mode: the paper's 2D runs (Sec. 2:
eight neighbouring bins in two dimensions; Sec. 4: equal-speed particles with
random directions between reflecting walls).

Checked against facts fixed outside the oracle: the scatter direction is a unit
vector uniform on the circle (norm, angle histogram, rejection rate pi/4); the
expected number of candidate pairs of a uniform planar gas in one step is the
two-dimensional collision-strip area C(N,2) 2 d0 <|g|> dt / A with <|g|> = 4s/pi
for equal speeds s in random directions; the cell search equals brute force;
each collision conserves momentum and energy to rounding and keeps the motion in
the plane; many collisions relax the speeds to the two-dimensional Maxwellian
(a Rayleigh law).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import kmc_inputs as ki
import oracle

U = 2.0 ** -53
NONE = 0xFFFFFFFF


def test_circle_vector_norm_and_isotropy():
    n = 60000
    vecs = np.empty((n, 3))
    tries = np.empty(n, dtype=np.int64)
    for i in range(n):
        v, t = oracle.circle_vector(9, 2000 + (i // 1000), i % 1000)
        vecs[i] = v
        tries[i] = t
    assert tries.min() >= 1
    assert np.all(vecs[:, 2] == 0.0)
    # two products, a difference or a doubling, one division per component
    norm2 = vecs[:, 0] ** 2 + vecs[:, 1] ** 2
    assert np.max(np.abs(norm2 - 1.0)) <= 8 * U
    # same rejection as the sphere: a point of the square accepted in the disk, pi/4
    acc = n / tries.sum()
    assert abs(acc - math.pi / 4) < 4 * math.sqrt(acc * (1 - acc) / tries.sum())
    from scipy.stats import chi2
    phi = np.arctan2(vecs[:, 1], vecs[:, 0]) / math.pi
    for comp in (phi, vecs[:, 0], vecs[:, 1]):
        # phi uniform; cos(phi) and sin(phi) follow the arcsine law on [-1, 1]
        if comp is phi:
            h, _ = np.histogram(comp, bins=20, range=(-1, 1))
            e = np.full(20, n / 20)
        else:
            edges = np.linspace(-1, 1, 21)
            cdf = 0.5 + np.arcsin(edges) / math.pi
            h, _ = np.histogram(comp, bins=edges)
            e = n * np.diff(cdf)
        stat = ((h - e) ** 2 / e).sum()
        assert stat < chi2.ppf(0.999, 19), stat
    assert np.all(np.abs(vecs[:, :2].mean(axis=0)) < 5 / math.sqrt(2 * n))


def test_circle_vector_is_the_doubled_disk_angle():
    """The accepted disk point's angle, doubled, is the direction: the planar draw and
    the spatial draw reject the same counters, so the attempt counts agree and the
    planar vector is (cos 2a, sin 2a) of the first accepted (u1, u2)."""
    for i in range(2000):
        v, t = oracle.circle_vector(3, 17, i)
        w, t3 = oracle.unit_vector(3, 17, i)
        assert t == t3
        # Marsaglia's sphere point has x = 2 u1 sqrt(1-s), y = 2 u2 sqrt(1-s): the
        # same (u1, u2) fixes its azimuth a = atan2(y, x); the planar vector is at 2a
        a = math.atan2(w[1], w[0])
        assert abs(v[0] - math.cos(2 * a)) < 1e-12 and abs(v[1] - math.sin(2 * a)) < 1e-12


def _planar_periodic(seed, n=4096, d0=0.002, dt=0.005):
    s = ki.equal_speed_setup(n=n, seed=seed, d0=d0, dt=dt)
    return s.with_(bc=(ki.PERIODIC, ki.PERIODIC, ki.REFLECT))


def test_planar_candidate_rate_step0_closed_form():
    """Candidates at step 0 of a uniform planar gas: C(N,2) * 2 d0 * <|g|> * dt / A,
    <|g|> = 2 s <|sin(theta/2)|> = 4 s / pi for equal speeds s, uniform theta;
    summed over independent seeds, within 3 sigma (Poisson)."""
    got = 0
    expect = 0.0
    for seed in range(300, 340):
        s = _planar_periodic(seed)
        st = oracle.State(ki.initial_state(s))
        pi, _, _, _ = oracle.candidate_pairs(s, st)
        got += len(pi)
        area = s.box[0] * s.box[1]
        expect += s.n * (s.n - 1) / 2 * 2 * s.d0 * (4 * 1.0 / math.pi) * s.dt / area
    sigma = math.sqrt(expect)
    assert abs(got - expect) < 3 * sigma, (got, expect, sigma)


@pytest.mark.parametrize("periodic", [False, True])
def test_planar_cell_search_equals_brute_force(periodic):
    s = ki.equal_speed_setup(n=3000, seed=21, d0=0.004, dt=0.01)
    if periodic:
        s = s.with_(bc=(ki.PERIODIC, ki.PERIODIC, ki.REFLECT))
    st = oracle.State(ki.initial_state(s))
    for _ in range(3):
        a = oracle.candidate_pairs(s, st, search=0)
        b = oracle.candidate_pairs(s, st, search=1)
        assert len(a[0]) > 0
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        oracle.run(s, st, 0, 7)


def test_planar_collisions_conserve_and_stay_in_plane():
    # periodic in x and y so that no wall reflection mixes into the velocity change
    s = _planar_periodic(5, d0=0.003, dt=0.01)
    st = oracle.State(ki.initial_state(s))
    z0 = st.a[2].copy()
    total = 0
    for step in range(6):
        before = [x.copy() for x in st.a]
        counts, partner, _ = oracle.step(s, st, step)
        total += counts["collisions"]
        assert np.all(st.a[5] == 0.0)
        assert np.array_equal(st.a[2], z0)
        for a in range(s.n):
            b = int(partner[a])
            if b == NONE or b < a:
                continue
            va = [before[3 + k][a] for k in range(2)]
            vb = [before[3 + k][b] for k in range(2)]
            wa = [st.a[3 + k][a] for k in range(2)]
            wb = [st.a[3 + k][b] for k in range(2)]
            vmax = max(math.hypot(*va), math.hypot(*vb))
            for k in range(2):
                dp = (Fraction(wa[k]) + Fraction(wb[k])) - (Fraction(va[k]) + Fraction(vb[k]))
                assert abs(float(dp)) <= 6 * U * vmax
            e0 = sum(Fraction(x) ** 2 for x in va + vb)
            e1 = sum(Fraction(x) ** 2 for x in wa + wb)
            assert abs(float(e1 - e0)) <= 16 * U * float(e0)
            # the pair's relative speed is unchanged (elastic), its direction is new
            g0 = math.hypot(va[0] - vb[0], va[1] - vb[1])
            g1 = math.hypot(wa[0] - wb[0], wa[1] - wb[1])
            assert abs(g1 - g0) <= 1e-12 * max(g0, 1.0)
    assert total > 300


def test_planar_gas_relaxes_to_two_dimensional_maxwellian():
    """Equal speeds relax under isotropic in-plane scattering to the 2D Maxwellian:
    speeds follow a Rayleigh law with sigma^2 = <v^2>/2 (energy fixed by the walls
    being elastic), each in-plane component is Gaussian."""
    from scipy import stats
    s = ki.equal_speed_setup(n=6000, seed=8, d0=0.006, dt=0.01)
    st = oracle.State(ki.initial_state(s))
    e0 = float((st.a[3] ** 2 + st.a[4] ** 2).sum())
    counts, _ = oracle.run(s, st, 0, 120)
    assert sum(c["collisions"] for c in counts) > 8 * s.n  # several collisions each
    v2 = st.a[3] ** 2 + st.a[4] ** 2
    assert abs(float(v2.sum()) - e0) < 1e-9 * e0
    sig = math.sqrt(float(v2.mean()) / 2)
    speed = np.sqrt(v2)
    assert stats.kstest(speed, stats.rayleigh(scale=sig).cdf).pvalue > 1e-3
    for k in (3, 4):
        assert stats.kstest(st.a[k], stats.norm(scale=sig).cdf).pvalue > 1e-3
    # equal speeds would fail: the initial state is far from the Rayleigh law
    st0 = ki.initial_state(s)
    sp0 = np.hypot(st0[3], st0[4])
    assert stats.kstest(sp0, stats.rayleigh(scale=sig).cdf).pvalue < 1e-10
