"""The allocation-free profile entry point (sim_profile_static) agrees with the
profile observable of a simulation (KMC_OBS_PROFILES), on two calls in a row.

sim_profile_static serves callers that cannot allocate device memory (an
application whose pool allocator owns the device memory, an in-situ hook inside
another code's time loop); its only scratch is a fixed array inside the library.
The second call checks that the counters left behind by the first call are cleared.
This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

import kmc_inputs as ki
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1310_3437_gb300 as kmc  # noqa: E402

U = 2.0 ** -53


def _entry():
    f = kmc.lib().sim_profile_static
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_int32,
                  C.c_double, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def _tolerance(ref):
    # the bound the profile parity tests use: (count + 2) u sum|terms| + count 2^-64 + 2 u |value|
    cnt = ref[:, 0]
    tol = np.zeros_like(ref)
    for q in range(1, 7):
        sq = ref[:, 4 + (q - 1) % 3]
        abs_sum = np.sqrt(np.maximum(cnt * sq, 0)) if q <= 3 else sq
        tol[:, q] = (cnt + 2) * U * abs_sum + cnt * 2.0 ** -64 + 2 * U * np.abs(ref[:, q])
    return tol


def test_static_profile_matches_the_profile_observable_twice():
    """Bit for bit the simulation's own profile (both use the same order-free
    fixed-point sums), and within the summation bound the oracle's id-order binary64
    profile of the same state, on two calls in a row."""
    setup = ki.piston_setup(n=1 << 14, seed=21, box=(8.0, 0.125, 0.125), profile_bins=256,
                            profile_every=1)
    arrays = ki.initial_state(setup)
    st = oracle.State(arrays)
    sim = kmc.Simulation(kmc.params_from_setup(setup, precision=kmc.KMC_GUARDED_FP32), arrays)
    f = _entry()
    n = setup.n
    stream = torch.cuda.current_stream()
    state = torch.empty(52 * n, dtype=torch.uint8, device="cuda")
    out = torch.empty(256 * 7, dtype=torch.float64, device="cuda")
    step = 0
    for call in range(2):
        sim.step(3).sync()
        for _ in range(3):
            _, _, oprof = oracle.step(setup, st, step)
            step += 1
        ref = sim.profiles()[-1]  # profile after the last of these steps
        sim.state_device(state)
        torch.cuda.synchronize()
        base = state.data_ptr()
        x, vx, vy, vz = (base + 8 * n * k for k in (0, 3, 4, 5))
        out.fill_(float("nan"))
        rc = f(x, vx, vy, vz, n, 256, setup.profile_range, out.data_ptr(), stream.cuda_stream)
        assert rc == kmc.KMC_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(256, 7)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), f"call {call}"
        assert np.array_equal(got[:, 0], oprof[:, 0]), f"call {call}: counts differ"
        assert np.all(np.abs(got - oprof) <= _tolerance(oprof)), f"call {call}: sums differ"
        assert got[:, 0].sum() == n
    sim.close()


def test_static_profile_of_a_too_fast_particle():
    """A velocity component whose square is beyond the fixed point (>= 2^31) turns its
    bin's six sums to NaN and leaves the other bins as the oracle's sums have them."""
    f = _entry()
    rng = np.random.default_rng(22)
    n = 5000
    x = rng.random(n)
    v = [rng.normal(0, 1, n) for _ in range(3)]
    v[2][17] = -6.0e4
    dev = [torch.from_numpy(a).cuda() for a in [x] + v]
    out = torch.empty(32 * 7, dtype=torch.float64, device="cuda")
    rc = f(*(d.data_ptr() for d in dev), n, 32, 1.0, out.data_ptr(), None)
    assert rc == kmc.KMC_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(32, 7)
    fast = int(x[17] * 32)
    want = np.zeros((32, 7))
    for i in range(n):  # plain sums in id order
        b = int(x[i] * 32)
        want[b, 0] += 1
        for a in range(3):
            want[b, 1 + a] += v[a][i]
            want[b, 4 + a] += v[a][i] * v[a][i]
    assert np.array_equal(got[:, 0], want[:, 0])
    assert np.isnan(got[fast, 1:]).all()
    ok = np.arange(32) != fast
    assert not np.isnan(got[ok]).any()
    assert np.all(np.abs(got[ok] - want[ok]) <= _tolerance(want[ok]))


def test_static_profile_rejects_bad_arguments():
    f = _entry()
    out = torch.empty(512 * 7, dtype=torch.float64, device="cuda")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    assert f(p, p, p, p, 4, 300, 1.0, out.data_ptr(), None) == kmc.KMC_EINVAL
    assert f(p, p, p, p, 4, 0, 1.0, out.data_ptr(), None) == kmc.KMC_EINVAL
    assert f(p, p, p, p, 4, 16, 0.0, out.data_ptr(), None) == kmc.KMC_EINVAL
    # n at or above 2^31: rejected before any array is read
    assert f(p, p, p, p, 1 << 31, 16, 1.0, out.data_ptr(), None) == kmc.KMC_EINVAL
    # host memory
    h = np.zeros(4)
    assert f(h.ctypes.data, p, p, p, 4, 16, 1.0, out.data_ptr(), None) == kmc.KMC_EINVAL
    assert f(p, p, p, p, 4, 16, 1.0, h.ctypes.data, None) == kmc.KMC_EINVAL
    torch.cuda.synchronize()
