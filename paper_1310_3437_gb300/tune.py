"""Autotuner for the knobs that change the work of a step but never its result.

Knobs: the search kernel (one warp per cell, one lane per particle over whole
stencil rows, one thread per particle cell by cell, or the per-step automatic
switch), the stencil (27 cells of width h, or 125 cells of width h/2), the
cell-size multiplier (>= 1: larger cells hold more particles) and how far the speed
split may thin out the slow grid.  Every combination yields bit-identical
trajectories (the tests check this), so the tuner only has to time them: it runs a
few steps of each candidate from the same initial state, times them with CUDA
events on the simulation's stream and keeps the fastest.  Choices are cached by
(precision, size bucket, occupancy bucket).
"""
from __future__ import annotations

import json
import math
import os

from .sim import Simulation, params_from_setup

DEFAULT_CANDIDATES = [
    # (search_kernel, stencil, cell_scale, split_min_occ): kernels 0 auto, 1 particle,
    # 2 cell, 3 row; split_min_occ = smallest mean slow-cell occupancy a speed split
    # may leave (0: no floor, 1e9: no split)
    (0, 1, 1.0, 0.0), (0, 1, 1.0, 2.0), (0, 1, 1.0, 4.0), (0, 1, 1.0, 8.0),
    (0, 1, 1.0, 1e9), (2, 1, 1.0, 1e9), (2, 1, 1.0, 16.0), (2, 1, 1.0, 8.0),
    (2, 1, 1.0, 5.0), (2, 1, 1.0, 3.0), (3, 1, 1.0, 0.0), (0, 2, 1.0, 0.0),
    (1, 1, 1.0, 0.0),
]


def occupancy_estimate(setup) -> float:
    """Mean particles per cell of width d0 + 2 v dt with v = 6 sqrt(kT/m) (order of the
    largest thermal speed), the grid the step starts from."""
    vol = float(setup.box[0]) * float(setup.box[1]) * float(setup.box[2])
    h = float(setup.d0) + 2.0 * 6.0 * float(setup.dt)
    return setup.n / vol * h ** 3


def bucket(setup, precision) -> str:
    nb = int(round(math.log2(max(1, setup.n))))
    ob = int(round(math.log2(max(1e-3, occupancy_estimate(setup))) * 2))
    return f"p{precision}_n{nb}_o{ob}"


class Autotuner:
    def __init__(self, cache_path: str | None = None, candidates=None, steps: int = 4,
                 warmup: int = 2):
        self.cache_path = cache_path
        self.candidates = list(candidates or DEFAULT_CANDIDATES)
        self.steps = steps
        self.warmup = warmup
        self.cache = {}
        self.trials = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def choose(self, setup, arrays, precision, stream=None) -> dict:
        """Best knobs for this set-up (timed once per bucket, then cached)."""
        key = bucket(setup, precision)
        if key in self.cache:
            return self.cache[key]
        import torch

        st = torch.cuda.Stream() if stream is None else stream
        results = []
        for kern, stencil, scale, occ in self.candidates:
            params = params_from_setup(setup, precision=precision, stencil=stencil,
                                       cell_scale=scale, search_kernel=kern, split_min_occ=occ)
            sim = Simulation(params, arrays, stream=st.cuda_stream)
            sim.step(self.warmup).sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            sim.step(self.steps)
            e1.record(st)
            e1.synchronize()
            sim.sync()
            ms = e0.elapsed_time(e1) / self.steps
            sim.close()
            results.append((ms, kern, stencil, scale, occ))
        results.sort()
        ms, kern, stencil, scale, occ = results[0]
        best = {"search_kernel": kern, "stencil": stencil, "cell_scale": scale,
                "split_min_occ": occ, "ms_per_step": ms}
        self.cache[key] = best
        self.trials[key] = [{"ms_per_step": r[0], "search_kernel": r[1], "stencil": r[2],
                             "cell_scale": r[3], "split_min_occ": r[4]} for r in results]
        if self.cache_path:
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1)
        return best

    def params(self, setup, arrays, precision, stream=None, **kw):
        best = self.choose(setup, arrays, precision, stream)
        return params_from_setup(setup, precision=precision, stencil=best["stencil"],
                                 cell_scale=best["cell_scale"],
                                 search_kernel=best["search_kernel"],
                                 split_min_occ=best["split_min_occ"], **kw)
