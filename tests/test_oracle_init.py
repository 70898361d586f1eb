"""Pins of the oracle's Philox-based initial states (the library's device-side
initialisation) and of its own logarithm.

Checked against facts fixed outside the oracle: libm's log (the oracle's log uses
only +, -, *, / and must stay within a few units of rounding of it); the laws the
states must follow (uniform positions on the 2^-53 grid, Gaussian components and
chi-square(3) speeds, one speed with isotropic directions, the blast's hot sphere);
and the per-particle keying (any subset of ids reproduces the full arrays).
"""
import math

import numpy as np
import pytest
from scipy import stats

import kmc_inputs as ki
import oracle

U = 2.0 ** -53


def test_log_matches_libm_within_rounding():
    rng = np.random.default_rng(3)
    # the polar method's s = u1^2 + u2^2 (u on the 2^-31 grid), values near 1 and a wide
    # range of magnitudes
    w = rng.integers(0, 2 ** 32, size=(2, 200000), dtype=np.uint64).astype(np.float64)
    u = w * 2.0 ** -31 - 1.0
    s = u[0] ** 2 + u[1] ** 2
    s = s[(s > 0) & (s < 1)]
    near1 = 1.0 - rng.random(20000) * 1e-6
    wide = np.exp2(rng.uniform(-62, 60, 50000))
    for x in (s, near1, wide, np.array([0.5, 2.0, 1.0 / 3.0, float.fromhex("0x1.6a09e667f3bcdp+0"),
                                        np.nextafter(float.fromhex("0x1.6a09e667f3bcdp+0"), 2.0), 2.0 ** -62])):
        got = oracle.log(x)
        want = np.log(x)
        err = np.abs(got - want)
        # a few roundings of the result's size (e ln2 product and sum, the series)
        tol = 4 * U * np.abs(want) + 2 * U * np.abs(np.floor(np.log2(x)) * math.log(2))
        assert np.all(err <= tol + 1e-300), (x[np.argmax(err - tol)], err.max())
    assert oracle.log(1.0) == 0.0
    assert oracle.log(0.5) == -float.fromhex("0x1.62e42fefa39efp-1")


def _spec_setups():
    return [ki.equilibrium_setup(n=60000, seed=21),
            ki.piston_setup(n=60000, seed=22, box=(8.0, 0.25, 0.25)),
            ki.equal_speed_setup(n=60000, seed=23, planar=False),
            ki.equal_speed_setup(n=60000, seed=24, planar=True)]


@pytest.mark.parametrize("k", range(4))
def test_positions_uniform_on_the_53_bit_grid(k):
    s = _spec_setups()[k]
    a = oracle.init_particles(s, ki.init_spec(s))
    for ax in range(3):
        x = a[ax]
        L = s.box[ax]
        if s.planar and ax == 2:
            assert np.all(x == 0.5 * L)
            continue
        assert np.all((x >= 0.0) & (x < L))
        assert stats.kstest(x / L, "uniform").pvalue > 1e-4
        if L == 1.0:  # x = u exactly: a multiple of 2^-53
            assert np.all(np.floor(x * 2.0 ** 53) == x * 2.0 ** 53)


@pytest.mark.parametrize("seed", [31, 32])
def test_maxwellian_components_and_speeds(seed):
    s = ki.equilibrium_setup(n=100000, seed=seed)
    a = oracle.init_particles(s, {"kind": 1, "sigma": 1.7})
    v = np.stack(a[3:6])
    for k in range(3):
        assert stats.kstest(v[k], stats.norm(scale=1.7).cdf).pvalue > 1e-4
    c = np.corrcoef(v)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 5 / math.sqrt(s.n))
    q = (v ** 2).sum(axis=0) / 1.7 ** 2
    assert stats.kstest(q, stats.chi2(3).cdf).pvalue > 1e-4
    # fourth moment of a Gaussian: 3 sigma^4 (a wrong log or sqrt would bend it)
    m4 = float((v[0] ** 4).mean()) / 1.7 ** 4
    assert abs(m4 - 3.0) < 6 * math.sqrt(96.0 / s.n)


def test_planar_maxwellian_has_two_components():
    s = ki.equal_speed_setup(n=80000, seed=33)
    a = oracle.init_particles(s, {"kind": 1, "sigma": 1.0})
    assert np.all(a[5] == 0.0)
    sp2 = a[3] ** 2 + a[4] ** 2
    assert stats.kstest(sp2, stats.chi2(2).cdf).pvalue > 1e-4


@pytest.mark.parametrize("planar", [False, True])
def test_equal_speed_directions(planar):
    s = ki.equal_speed_setup(n=80000, seed=34, planar=planar, speed=2.5)
    a = oracle.init_particles(s, ki.init_spec(s))
    v = np.stack(a[3:6])
    sp = np.sqrt((v ** 2).sum(axis=0))
    assert np.max(np.abs(sp - 2.5)) <= 8 * U * 2.5
    if planar:
        assert np.all(v[2] == 0.0)
        phi = np.arctan2(v[1], v[0])
        assert stats.kstest(phi, stats.uniform(loc=-math.pi, scale=2 * math.pi).cdf).pvalue > 1e-4
    else:
        # Archimedes: each component of a uniform direction is uniform in [-1, 1]
        for k in range(3):
            assert stats.kstest(v[k] / 2.5, stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-4


def test_blast_hot_sphere():
    s = ki.blast_setup(n=300000, seed=35)
    spec = ki.init_spec(s)
    a = oracle.init_particles(s, spec)
    x = np.stack(a[:3])
    c = np.array(spec["center"])[:, None]
    r2 = ((x - c) ** 2).sum(axis=0)
    hot = np.arange(s.n) < spec["n_hot"]
    assert np.array_equal(r2 < spec["radius"] ** 2, hot)
    # uniform in the ball: (r/R)^3 uniform in [0, 1)
    q = (np.sqrt(r2[hot]) / spec["radius"]) ** 3
    assert stats.kstest(q, "uniform").pvalue > 1e-4
    # outside: uniform in the box minus the ball, e.g. the corner octant [0, 0.25)^3
    # holds its volume share
    cold = ~hot
    corner = np.all(x[:, cold] < 0.25, axis=0).sum()
    vol = 1.0 - 4.0 / 3.0 * math.pi * spec["radius"] ** 3
    e = cold.sum() * 0.25 ** 3 / vol
    assert abs(corner - e) < 4 * math.sqrt(e)
    v = np.stack(a[3:6])
    assert stats.kstest(v[0, hot], stats.norm(scale=10.0).cdf).pvalue > 1e-4
    assert stats.kstest(v[1, cold], stats.norm(scale=1.0).cdf).pvalue > 1e-4


def test_any_subset_of_ids_reproduces_the_full_arrays():
    for s in _spec_setups()[:3] + [ki.blast_setup(n=50000, seed=36)]:
        spec = ki.init_spec(s)
        full = oracle.init_particles(s, spec)
        ids = np.random.default_rng(1).choice(s.n, 777, replace=False).astype(np.uint32)
        part = oracle.init_particles(s, spec, ids)
        for k in range(6):
            assert np.array_equal(part[k], full[k][ids])
        # and another seed gives other arrays
        other = oracle.init_particles(s.with_(seed=s.seed + 1000), spec, ids)
        assert not np.array_equal(other[0], part[0])
