"""The paper's timing workloads at their stated sizes (Fig. 1: 10^8 particles in
3D; Fig. 3: 4 x 10^7 in 2D), checked through properties that hold at any size: the
oracle cannot step them in seconds.  One speed, reflecting walls: every collision
conserves energy to rounding and a wall reflection flips a component exactly, so
the total kinetic energy stays n s^2 / 2; the planar gas stays in its plane; every
particle stays in the box; the first steps collide at the rate the mean free path
sets."""
import math

import numpy as np
import pytest

import kmc_inputs as ki

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1310_3437_gb300 as kmc  # noqa: E402


@pytest.mark.parametrize("figure", [1, 3])
def test_paper_workload_invariants_at_full_size(figure):
    s = ki.paper_timing_setup(figure)
    sim = kmc.Simulation(kmc.params_from_setup(s, precision=kmc.KMC_GUARDED_FP32),
                         init=ki.init_spec(s))
    steps = 4
    sim.step(steps).sync()
    counts = sim.counts()
    buf = torch.empty(52 * s.n, dtype=torch.uint8, device="cuda")
    sim.state_device(buf)
    torch.cuda.synchronize()
    f = buf[: 48 * s.n].view(torch.float64).view(6, s.n)
    v2 = (f[3] * f[3] + f[4] * f[4] + f[5] * f[5]).sum().item()
    # energy: n s^2 (s = 1) up to the rounding of the collisions and of the sum
    assert abs(v2 - s.n) < 1e-9 * s.n, v2
    for a in range(3):
        assert bool((f[a] >= 0).all()) and bool((f[a] <= s.box[a]).all())
    if s.planar:
        assert bool((f[5] == 0).all())
        assert bool((f[2] == 0.5 * s.box[2]).all())
    # collisions per step: n nu dt / 2 with nu = 1/(sqrt2 lambda) * <g> (3D, <g> = 4/3)
    # or n 2 d0 <g> (2D, <g> = 4/pi), less what mutual matching leaves unmatched
    if s.planar:
        nu = s.n * 2.0 * s.d0 * 4.0 / math.pi
    else:
        nu = s.n * math.pi * s.d0 ** 2 * 4.0 / 3.0
    expect = s.n * nu * s.dt / 2.0
    coll = np.mean([c["collisions"] for c in counts])
    assert 0.8 * expect < coll < 1.02 * expect, (coll, expect)
    sim.close()
