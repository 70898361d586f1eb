"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* Philox4x32-10: the published known-answer vectors and an independent library
  implementation (Triton's Philox, run by its CPU interpreter).
* Marsaglia sphere point: unit norm within rounding, isotropy (chi-square).
* Candidate test (Sec. 2, three criteria): closest approach found by sampling the
  straight-line trajectory; the accepted set of separations is a cylinder of volume
  pi d0^2 |v| dt (Monte Carlo); bitwise symmetry of the pair key.
* Cell search == O(N^2) brute force (the paper's claim that the neighbourhood
  search finds the closest partner without scanning the whole space).
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import kmc_inputs as ki
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert oracle.philox4x32_10(ctr, key).tolist() == want


_TRITON_SCRIPT = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(ctr_ptr, out_ptr, seed, BLOCK: tl.constexpr):
    offs = tl.arange(0, BLOCK)
    c0 = tl.load(ctr_ptr + 0 * BLOCK + offs)
    c1 = tl.load(ctr_ptr + 1 * BLOCK + offs)
    c2 = tl.load(ctr_ptr + 2 * BLOCK + offs)
    c3 = tl.load(ctr_ptr + 3 * BLOCK + offs)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 0 * BLOCK + offs, r0)
    tl.store(out_ptr + 1 * BLOCK + offs, r1)
    tl.store(out_ptr + 2 * BLOCK + offs, r2)
    tl.store(out_ptr + 3 * BLOCK + offs, r3)

data = np.load(sys.argv[1])
ctr = torch.from_numpy(data["ctr"].astype(np.int64)).to(torch.uint32)
out = torch.zeros_like(ctr)
k[(1,)](ctr, out, int(data["seed"]), BLOCK=ctr.shape[1])
np.save(sys.argv[2], out.to(torch.int64).numpy() & 0xFFFFFFFF)
"""


def test_philox_matches_triton_interpreter(tmp_path):
    """Triton's own Philox (CPU interpreter) is an implementation independent of ours."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(12345)
    for trial in range(2):
        ctr = rng.integers(0, 2 ** 32, size=(4, 64), dtype=np.uint64).astype(np.uint32)
        seed = int(rng.integers(0, 2 ** 63)) | (trial << 63)
        inp = tmp_path / f"in{trial}.npz"
        outp = tmp_path / f"out{trial}.npy"
        np.savez(inp, ctr=ctr, seed=np.uint64(seed))
        env = dict(os.environ, TRITON_INTERPRET="1")
        r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT, str(inp), str(outp)],
                           env=env, capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            pytest.skip(f"triton interpreter unavailable: {r.stderr[-300:]}")
        ref = np.load(outp).astype(np.uint64)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for lane in range(ctr.shape[1]):
            got = oracle.philox4x32_10(ctr[:, lane], key)
            assert got.astype(np.uint64).tolist() == ref[:, lane].tolist()


def test_unit_vector_norm_and_isotropy():
    n = 60000
    vecs = np.empty((n, 3))
    tries = np.empty(n, dtype=np.int64)
    for i in range(n):
        v, t = oracle.unit_vector(7, 1000 + (i // 1000), i % 1000)
        vecs[i] = v
        tries[i] = t
    assert tries.min() >= 1
    # |n|^2 - 1 within a few units of rounding (three products, one sqrt, sums)
    norm2 = (vecs ** 2).sum(axis=1)
    assert np.max(np.abs(norm2 - 1.0)) <= 8 * U
    # Marsaglia acceptance rate is pi/4 per attempt
    acc = n / tries.sum()
    assert abs(acc - math.pi / 4) < 4 * math.sqrt(acc * (1 - acc) / tries.sum())
    # isotropy: cos(theta) = z uniform in [-1, 1], phi uniform; chi-square with 20 bins
    from scipy.stats import chi2
    for comp in (vecs[:, 2], vecs[:, 0], np.arctan2(vecs[:, 1], vecs[:, 0]) / math.pi):
        h, _ = np.histogram(comp, bins=20, range=(-1, 1))
        e = n / 20
        stat = ((h - e) ** 2 / e).sum()
        assert stat < chi2.ppf(0.999, 19)
    assert np.all(np.abs(vecs.mean(axis=0)) < 5 / math.sqrt(3 * n))


def _two_particle_state(ri, rj, vi, vj):
    arr = [np.array([ri[k], rj[k]]) for k in range(3)] + [np.array([vi[k], vj[k]]) for k in range(3)]
    return oracle.State(arr)


def test_pair_key_matches_sampled_trajectory():
    """t* and d_min from the oracle agree with the minimum of |r + v t| found by
    dense sampling of the straight-line relative trajectory."""
    rng = np.random.default_rng(3)
    setup = ki.Setup(n=2, box=(100.0, 100.0, 100.0), bc=(1, 1, 1), d0=0.3, dt=1.0)
    hits = 0
    for _ in range(150):
        ri = rng.uniform(40, 60, 3)
        rj = ri + rng.normal(0, 0.4, 3)
        vi = rng.normal(0, 1, 3)
        vj = rng.normal(0, 1, 3)
        st = _two_particle_state(ri, rj, vi, vj)
        ok, d2, t = oracle.pair(setup, st, 0, 1)
        r = rj - ri
        v = vj - vi
        ts = np.linspace(-3, 3, 600001)
        dist2 = ((r[None, :] + ts[:, None] * v[None, :]) ** 2).sum(axis=1)
        k = int(np.argmin(dist2))
        t_s, d2_s = ts[k], dist2[k]
        expect = (0 <= t_s < setup.dt) and (d2_s < setup.d0 ** 2)
        margin = (abs(t_s) < 2e-5 or abs(t_s - setup.dt) < 2e-5
                  or abs(d2_s - setup.d0 ** 2) < 1e-9)
        if not margin:
            assert ok == expect
        if ok:
            hits += 1
            assert abs(t - t_s) < 2e-5
            assert abs(d2 - d2_s) < 1e-9 + 1e-6 * d2_s
    assert hits > 8


def test_pair_key_bitwise_symmetric_and_min_image():
    rng = np.random.default_rng(4)
    L = 1.0
    setup = ki.Setup(n=2, box=(L, L, L), bc=(0, 0, 0), d0=0.2, dt=0.5)
    found = 0
    for _ in range(3000):
        ri = rng.uniform(0, L, 3)
        # partner near, possibly across the periodic boundary
        rj = np.mod(ri + rng.normal(0, 0.1, 3), L)
        rj = np.minimum(rj, np.nextafter(L, 0))
        vi = rng.normal(0, 1, 3)
        vj = rng.normal(0, 1, 3)
        st = _two_particle_state(ri, rj, vi, vj)
        a = oracle.pair(setup, st, 0, 1)
        b = oracle.pair(setup, st, 1, 0)
        assert a[0] == b[0]
        if a[0]:
            found += 1
            assert a[1] == b[1] and a[2] == b[2]  # bitwise identical keys
        # the same geometry translated so that no boundary is crossed gives the
        # same verdict (minimum image)
        shift = 0.5 * L - ri
        rj2 = ri + shift + ((rj - ri + 0.5 * L) % L - 0.5 * L)
        st2 = _two_particle_state(ri + shift, rj2, vi, vj)
        c = oracle.pair(ki.Setup(n=2, box=(10, 10, 10), bc=(1, 1, 1), d0=0.2, dt=0.5), st2, 0, 1)
        if abs(np.abs(rj - ri).max() - 0.5 * L) > 1e-6:
            assert c[0] == a[0]
    assert found > 50


def test_candidate_region_is_a_cylinder():
    """For fixed relative velocity v, the separations r that pass the test fill a
    cylinder of radius d0 and length |v| dt: volume pi d0^2 |v| dt."""
    rng = np.random.default_rng(5)
    d0, dt = 0.05, 0.1
    setup = ki.Setup(n=2, box=(10, 10, 10), bc=(1, 1, 1), d0=d0, dt=dt)
    v = np.array([0.7, -0.2, 0.4])
    box = 0.2
    m = 60000
    hit = 0
    for _ in range(m):
        r = rng.uniform(-box / 2, box / 2, 3)
        st = _two_particle_state(np.array([5.0, 5.0, 5.0]), 5.0 + r, np.zeros(3), v)
        hit += oracle.pair(setup, st, 0, 1)[0]
    p = math.pi * d0 * d0 * np.linalg.norm(v) * dt / box ** 3
    assert abs(hit / m - p) < 4 * math.sqrt(p * (1 - p) / m)


def _random_states():
    out = []
    s = ki.equilibrium_setup(n=3000, seed=11, d0=0.03, dt=0.02)
    out.append((s, oracle.State(ki.initial_state(s))))
    s = ki.piston_setup(n=4000, seed=12, box=(2.0, 0.5, 0.5), lam=0.02)
    out.append((s, oracle.State(ki.initial_state(s))))
    # clustered particles with many equal velocities and positions near the walls
    rng = np.random.default_rng(13)
    n = 1500
    pos = [np.minimum(np.abs(rng.normal(0, 0.02, n)) % 1.0, np.nextafter(1.0, 0)) for _ in range(3)]
    pos[1][:200] = np.nextafter(1.0, 0)
    pos[0][200:400] = 0.0
    vel = [np.round(rng.normal(0, 1, n), 1) for _ in range(3)]
    s = ki.Setup(n=n, box=(1.0, 1.0, 1.0), bc=(0, 0, 0), d0=0.01, dt=0.01, seed=13,
                 name="equilibrium_adversarial")
    out.append((s, oracle.State(pos + vel)))
    # a thin periodic slab: y and z collapse to one cell
    s = ki.Setup(n=2000, box=(1.0, 0.05, 0.05), bc=(0, 0, 0), d0=0.01, dt=0.01, seed=14,
                 name="equilibrium_slab")
    rng = np.random.default_rng(14)
    pos = [rng.random(n := 2000) * b for b in (1.0, 0.05, 0.05)]
    vel = [rng.normal(0, 1, n) for _ in range(3)]
    out.append((s, oracle.State(pos + vel)))
    return out


def test_cell_search_equals_brute_force():
    for setup, st in _random_states():
        a = oracle.candidate_pairs(setup, st, search=0)
        b = oracle.candidate_pairs(setup, st, search=1)
        assert len(a[0]) > 0
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        # also after some steps (last-partner exclusions present, walls hit)
        st2 = st.copy()
        oracle.run(setup, st2, 0, 5)
        a = oracle.candidate_pairs(setup, st2, search=0)
        b = oracle.candidate_pairs(setup, st2, search=1)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_threads_do_not_change_results():
    s = ki.equilibrium_setup(n=4096, seed=21)
    a = oracle.State(ki.initial_state(s))
    b = a.copy()
    ca, _ = oracle.run(s, a, 0, 10, threads=1)
    cb, _ = oracle.run(s, b, 0, 10, threads=4)
    assert ca == cb
    for x, y in zip(a.a, b.a):
        assert np.array_equal(x, y)
    assert np.array_equal(a.last, b.last)


def test_vmax2_is_the_largest_squared_speed():
    """The oracle's largest squared speed (the maximum speed that Sec. 2 derives the
    time step from) against exact rational arithmetic: every square and sum computed
    exactly, the maximum taken exactly, then compared within the three roundings of
    (vx*vx + vy*vy) + vz*vz.  A (3, 4, 12) particle has |v|^2 = 169 exactly."""
    from fractions import Fraction

    rng = np.random.default_rng(71)
    for n in (1, 2, 7, 1000):
        v = [rng.normal(0, 1, n) * 3 for _ in range(3)]
        want = max(sum(Fraction(float(c[i])) ** 2 for c in v) for i in range(n))
        st = oracle.State([np.zeros(n)] * 3 + v)
        got = oracle.vmax2(st)
        assert abs(Fraction(got) - want) <= want * Fraction(3 * U)
    v = [np.array([0.5, 3.0, -1.0]), np.array([0.5, -4.0, 2.0]), np.array([0.5, 12.0, 2.0])]
    st = oracle.State([np.zeros(3)] * 3 + v)
    assert oracle.vmax2(st) == 169.0
    # the largest particle wins wherever it sits, whichever component carries it
    for pos in range(3):
        for comp in range(3):
            v = [np.full(4, 0.25) for _ in range(3)]
            v[comp][pos] = -7.0
            st = oracle.State([np.zeros(4)] * 3 + v)
            assert oracle.vmax2(st) == 49.0 + 2 * 0.0625
