"""Observables and failure paths of the C ABI on the GPU.

* KMC_OBS_VMAX (Sec. 2: the time step and, here, the cell size come from the largest
  particle speed; Sec. 4 reduces it over all domains) equals the oracle's
  sqrt(max |v|^2) bit for bit, over the particles still in the gas.
* A profile bin holding a particle too fast for the fixed-point sums reports NaN
  sums for that bin only; every other bin and every count stays as before.
* A simulation that does not fit in device memory fails with KMC_ENOMEM, frees what
  it allocated, and the device keeps working.
"""
import ctypes as C
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

U = 2.0 ** -53


def _live_vmax(st):
    live = st.last != oracle.ABSORBED
    sub = oracle.State([a[live] for a in st.a])
    return math.sqrt(oracle.vmax2(sub)) if live.any() else 0.0


@pytest.mark.parametrize("precision", [kmc.KMC_FP64, kmc.KMC_GUARDED_FP32])
def test_vmax_observable_equals_the_oracle(precision):
    s = ki.piston_setup(n=1 << 14, seed=51, box=(8.0, 0.125, 0.125), profile_bins=0,
                        profile_every=0)
    arrays = ki.initial_state(s)
    st = oracle.State(arrays)
    sim = kmc.Simulation(kmc.params_from_setup(s, precision=precision), arrays)
    assert sim.vmax() == _live_vmax(st)
    oracle.run(s, st, 0, 40)  # the piston adds 2 u_p to every particle it reflects
    sim.step(40).sync()
    assert sim.vmax() == _live_vmax(st)
    # device destination
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert kmc.sim_observe(sim.handle, kmc.KMC_OBS_VMAX, out.data_ptr(), 8) == 1
    assert out.item() == _live_vmax(st)
    sim.close()


def test_vmax_observable_skips_absorbed_particles():
    s = ki.equilibrium_setup(n=3000, seed=52, L=0.5, d0=0.002)
    s = s.with_(bc=(kmc.KMC_ABSORB, kmc.KMC_PERIODIC, kmc.KMC_ABSORB), piston_x0=0.5)
    arrays = ki.initial_state(s)
    arrays[0][7], arrays[3][7] = 0.499, 40.0  # leaves through the upper x wall at once
    st = oracle.State(arrays)
    sim = kmc.Simulation(kmc.params_from_setup(s, precision=kmc.KMC_GUARDED_FP32), arrays)
    assert sim.vmax() == _live_vmax(st) >= 40.0
    oc, _ = oracle.run(s, st, 0, 30)
    sim.step(30).sync()
    assert st.last[7] == oracle.ABSORBED and sum(c["absorbed"] for c in oc) > 100
    assert sim.vmax() == _live_vmax(st) < 40.0
    sim.close()


def test_profile_bins_of_too_fast_particles_are_nan():
    """vy = 9e4 (vy^2 = 8.1e9 >= 2^31, beyond the three 32-bit digits of the fixed-point
    sums): the bins holding a particle with |v_a| >= 2^31 or v_a^2 >= 2^31 after a step
    (taken from the oracle's state, collisions share the energy out) report NaN for
    their six sums, the others agree with the oracle's sums."""
    s = ki.equilibrium_setup(n=4096, seed=53, dt=1e-6)
    s = s.with_(profile_bins=64, profile_every=1, profile_range=1.0)
    arrays = ki.initial_state(s)
    arrays[4][11] = 9.0e4
    st = oracle.State(arrays)
    steps = 4
    sim = kmc.Simulation(kmc.params_from_setup(s, precision=kmc.KMC_FP64), arrays)
    sim.step(steps).sync()
    gprof = sim.profiles()
    assert gprof.shape == (steps, 64, 7)
    for k in range(steps):
        _, _, oprof = oracle.step(s, st, k)
        v = np.stack(st.a[3:6])
        fast = ((np.abs(v) >= 2.0 ** 31) | (v * v >= 2.0 ** 31)).any(axis=0)
        want_nan = np.zeros(64, bool)
        want_nan[(st.a[0][fast] * 64).astype(int)] = True
        assert want_nan.any()
        assert np.array_equal(gprof[k, :, 0], oprof[:, 0])
        assert np.array_equal(np.isnan(gprof[k, :, 1:]).all(axis=1), want_nan), k
        assert not np.isnan(gprof[k, ~want_nan, 1:]).any()
        ok = ~want_nan
        cnt = oprof[ok, 0]
        for q in range(1, 7):
            sq = oprof[ok, 4 + (q - 1) % 3]
            abs_sum = np.sqrt(np.maximum(cnt * sq, 0)) if q <= 3 else sq
            tol = (cnt + 2) * U * abs_sum + cnt * 2.0 ** -64 + 2 * U * np.abs(oprof[ok, q])
            assert np.all(np.abs(gprof[k, ok, q] - oprof[ok, q]) <= tol), q
    sim.close()


def test_creation_beyond_device_memory_fails_cleanly():
    """2^31 - 4096 particles need well over the GPU's memory (about 400 B each): the
    allocation fails, KMC_ENOMEM comes back with a message, nothing is left
    allocated, and a simulation created next runs as usual.  The state would be drawn
    on the device, so no host array is ever read."""
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    s = ki.equilibrium_setup(n=0x7FFFF000, seed=54)
    p = kmc.params_from_setup(s, precision=kmc.KMC_FP64)
    assert kmc.sim_bytes_required(p) > free0
    init = kmc.init_from_spec(ki.init_spec(ki.equilibrium_setup(n=4096, seed=54)))
    out = C.c_void_p()
    rc = kmc.lib().sim_create_init(C.byref(p), C.byref(init), None, C.byref(out))
    assert rc == kmc.KMC_ENOMEM
    assert out.value is None
    assert "cudaMalloc" in kmc.sim_last_error(None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)
    small = ki.equilibrium_setup(n=4096, seed=54)
    arrays = ki.initial_state(small)
    st = oracle.State(arrays)
    oracle.run(small, st, 0, 5)
    sim = kmc.Simulation(kmc.params_from_setup(small, precision=kmc.KMC_FP64), arrays)
    sim.step(5).sync()
    got, last = sim.state()
    for k in range(6):
        assert np.array_equal(got[k], st.a[k])
    sim.close()


def test_bounded_scan_wait_reports_a_timeout_and_the_device_stays_usable():
    """The cell scan's tiles wait for their predecessors' sums with a bounded wait.  A
    test flag makes them wait for a status word that is never written: each wait runs
    out after about a second, the step is abandoned with the timeout status, sim_sync
    returns KMC_ETIMEOUT, and the next simulation on the device runs as usual."""
    # a tube whose key space spans many scan tiles (8192 keys each), so that tiles wait
    s = ki.piston_setup(n=1 << 17, seed=55, profile_bins=0, profile_every=0)
    arrays = ki.initial_state(s)
    p = kmc.params_from_setup(s, precision=kmc.KMC_FP64, flags=kmc.KMC_FLAG_SCAN_WAIT_TEST)
    sim = kmc.Simulation(p, arrays)
    sim.step(1)
    with pytest.raises(kmc.KmcError) as e:
        sim.sync()
    assert e.value.code == kmc.KMC_ETIMEOUT
    assert sim.counts() == []  # the abandoned step left no record
    sim.close()
    st = oracle.State(arrays)
    oracle.run(s, st, 0, 3)
    ok = kmc.Simulation(kmc.params_from_setup(s, precision=kmc.KMC_FP64), arrays).step(3).sync()
    assert ok.counts()[0]["cells"] > 4 * 8192  # several scan tiles, so tiles did wait
    got, _ = ok.state()
    for k in range(6):
        assert np.array_equal(got[k], st.a[k])
    ok.close()
