"""The allocation-free profile entry point (sim_profile_static) agrees with the
profile observable of a simulation (KMC_OBS_PROFILES), on two calls in a row.

sim_profile_static serves callers that cannot allocate device memory; its only
scratch is a fixed array inside the library.  The second call checks that the
counters left behind by the first call are cleared.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

import kmc_inputs as ki

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
    setup = ki.piston_setup(n=1 << 14, seed=21, box=(8.0, 0.125, 0.125), profile_bins=256,
                            profile_every=1)
    sim = kmc.Simulation(kmc.params_from_setup(setup, precision=kmc.KMC_GUARDED_FP32),
                         ki.initial_state(setup))
    f = _entry()
    n = setup.n
    stream = torch.cuda.current_stream()
    state = torch.empty(52 * n, dtype=torch.uint8, device="cuda")
    out = torch.empty(256 * 7, dtype=torch.float64, device="cuda")
    for call in range(2):
        sim.step(3).sync()
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
        assert np.array_equal(got[:, 0], ref[:, 0]), f"call {call}: counts differ"
        assert np.all(np.abs(got - ref) <= _tolerance(ref)), f"call {call}: sums differ"
        assert got[:, 0].sum() == n
    sim.close()


def test_static_profile_rejects_too_many_bins():
    f = _entry()
    out = torch.empty(512 * 7, dtype=torch.float64, device="cuda")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = f(x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 4, 300, 1.0, out.data_ptr(), None)
    assert rc == kmc.KMC_EINVAL
    rc = f(x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 4, 0, 1.0, out.data_ptr(), None)
    assert rc == kmc.KMC_EINVAL
