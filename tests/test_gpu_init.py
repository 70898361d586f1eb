"""Device-side initial states (sim_create_init) against the oracle's Philox
initialisation: the arrays must be bit-identical, at small sizes for every
particle and at the headline size for sampled ids, and the runs that start from
them must stay bit-identical to the oracle."""
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
NONE = 0xFFFFFFFF


def _same(a, b, what):
    a = np.asarray(a)
    b = np.asarray(b)
    if not np.array_equal(a.view(np.uint64), b.view(np.uint64)):
        bad = np.nonzero(a.view(np.uint64) != b.view(np.uint64))[0]
        raise AssertionError(f"{what}: {len(bad)} differ, first {bad[:5]}: {a[bad[:3]]} vs {b[bad[:3]]}")


def _setups():
    return [
        ki.equilibrium_setup(n=50001, seed=41),
        ki.piston_setup(n=65537, seed=42, box=(8.0, 0.25, 0.25), profile_bins=0, profile_every=0),
        ki.equal_speed_setup(n=40003, seed=43, planar=False, d0=0.004, dt=0.005),
        ki.equal_speed_setup(n=40003, seed=44, planar=True, d0=0.002, dt=0.005),
        ki.blast_setup(n=70001, seed=45, lam_bg=0.05, steps=20),
    ]


@pytest.mark.parametrize("k", range(5))
def test_device_init_equals_oracle_init(k):
    s = _setups()[k]
    spec = ki.init_spec(s)
    want = oracle.init_particles(s, spec)
    sim = kmc.Simulation(kmc.params_from_setup(s, precision=FP32), init=spec)
    got, last = sim.state()
    for c in range(6):
        _same(got[c], want[c], f"component {c}")
    assert np.all(last == NONE)
    sim.close()


def test_planar_maxwellian_and_other_seed():
    s = ki.equal_speed_setup(n=30011, seed=46, planar=True)
    spec = {"kind": kmc.KMC_INIT_MAXWELL, "sigma": 0.7}
    sim = kmc.Simulation(kmc.params_from_setup(s), init=spec)
    got, _ = sim.state()
    want = oracle.init_particles(s, spec)
    for c in range(6):
        _same(got[c], want[c], f"component {c}")
    assert np.all(got[5] == 0.0)
    s2 = s.with_(seed=47)
    got2, _ = kmc.Simulation(kmc.params_from_setup(s2), init=spec).state()
    assert not np.array_equal(got2[0], got[0])


@pytest.mark.parametrize("k,precision", [(0, FP32), (1, FP64), (3, FP32), (4, FP32)])
def test_runs_from_device_init_stay_bit_exact(k, precision):
    s = _setups()[k]
    spec = ki.init_spec(s)
    st = oracle.State(oracle.init_particles(s, spec))
    oc, _ = oracle.run(s, st, 0, 25)
    sim = kmc.Simulation(kmc.params_from_setup(s, precision=precision), init=spec)
    sim.step(25).sync()
    got, last = sim.state()
    for c in range(6):
        _same(got[c], st.a[c], f"component {c}")
    assert np.array_equal(last, st.last)
    gc = sim.counts()
    assert [c["collisions"] for c in gc] == [c["collisions"] for c in oc]
    assert sum(c["collisions"] for c in oc) > 100


def test_full_size_tube_device_init_sampled():
    """The 2^24-particle piston tube drawn on the device: sampled ids (and the first
    and last) equal the oracle's draws for those ids."""
    s = ki.piston_setup(n=1 << 24, seed=2, profile_bins=0, profile_every=0)
    spec = ki.init_spec(s)
    sim = kmc.Simulation(kmc.params_from_setup(s, precision=FP32), init=spec)
    buf = torch.empty(52 * s.n, dtype=torch.uint8, device="cuda")
    sim.state_device(buf)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    ids = np.unique(np.concatenate([rng.choice(s.n, 20000, replace=False), [0, 1, s.n - 1]]))
    ids = ids.astype(np.uint32)
    want = oracle.init_particles(s, spec, ids)
    f = buf[: 48 * s.n].view(torch.float64).view(6, s.n)
    idx = torch.from_numpy(ids.astype(np.int64)).to("cuda")
    for c in range(6):
        _same(f[c].index_select(0, idx).cpu().numpy(), want[c], f"component {c}")
    last = buf[48 * s.n:].view(torch.int32)
    assert bool((last == -1).all())
    sim.close()
