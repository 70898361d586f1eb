"""The autotuner's host side (no GPU): the occupancy estimate it buckets on, the bucket
keys, and a cached choice applied to the parameters without timing anything."""
import json
import math

import kmc_inputs as ki
import paper_1310_3437_gb300 as kmc
from paper_1310_3437_gb300 import tune


def test_occupancy_estimate_is_particles_per_cell_of_the_starting_grid():
    s = ki.piston_setup(n=1 << 20)
    vol = s.box[0] * s.box[1] * s.box[2]
    h = s.d0 + 12.0 * s.dt  # d0 + 2 v dt with v = 6 thermal speeds
    assert math.isclose(tune.occupancy_estimate(s), s.n / vol * h ** 3, rel_tol=1e-12)


def test_buckets_separate_sizes_and_precisions_and_join_neighbours():
    a = ki.piston_setup(n=1 << 20)
    assert tune.bucket(a, kmc.KMC_FP64) != tune.bucket(a, kmc.KMC_GUARDED_FP32)
    assert tune.bucket(a, kmc.KMC_FP64) != tune.bucket(ki.piston_setup(n=1 << 22), kmc.KMC_FP64)
    # a few percent more particles: the same size bucket and occupancy bucket
    b = ki.piston_setup(n=int((1 << 20) * 1.03))
    assert tune.bucket(a, kmc.KMC_FP64) == tune.bucket(b, kmc.KMC_FP64)


def test_a_cached_choice_is_applied_without_timing(tmp_path):
    s = ki.equilibrium_setup(n=5000, seed=3)
    key = tune.bucket(s, kmc.KMC_GUARDED_FP32)
    choice = {"search_kernel": 2, "stencil": 1, "cell_scale": 1.5, "split_min_occ": 8.0,
              "ms_per_step": 0.1}
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({key: choice}))
    t = tune.Autotuner(cache_path=str(path))
    assert t.choose(s, None, kmc.KMC_GUARDED_FP32) == choice  # no simulation is made
    p = t.params(s, None, kmc.KMC_GUARDED_FP32, history_cap=77)
    assert (p.search_kernel, p.stencil, p.cell_scale, p.split_min_occ) == (2, 1, 1.5, 8.0)
    assert p.history_cap == 77 and p.precision == kmc.KMC_GUARDED_FP32 and p.n == s.n
