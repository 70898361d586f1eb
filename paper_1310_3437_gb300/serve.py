"""Serving loop: simulation requests admitted by HBM budget and stepped together.

Requests arrive over time (each with its own parameters, initial state -- arrays,
or a descriptor of a state drawn on the device -- and step count).  The server admits queued requests in arrival order while their device
footprint (``sim_bytes_required``) fits the HBM budget, adds each admitted
simulation to one group with a step budget equal to its requested steps, and
advances the group in short bursts: one launch per kernel per step covers every
live simulation (members whose budget is spent are skipped on the device).  A
burst is at most ``burst_steps`` long and ends when the live request closest to its
end has run its steps, so no request waits for a burst to run past its end.  A
request is complete when its budget is spent and its final state and per-step
counts have been copied to the host; it then leaves the group and its memory is
freed, so queued requests can be admitted.  Latency is measured from arrival to
that point.  Nothing here touches simulation data: all of it runs in libkmc.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import KMC_GUARDED_FP32, sim_bytes_required
from .sim import Group, Simulation, params_from_setup


@dataclass
class Request:
    rid: int
    setup: object              # n, box, bc, d0, dt, seed, ... (see params_from_setup)
    steps: int
    arrival: float             # seconds after the start of the run
    arrays: object = None      # six float64 arrays, or a callable returning them
    init: dict = None          # or a kmc_init descriptor (dict): state drawn on the device
    precision: int = KMC_GUARDED_FP32
    # filled in by the server
    admitted: float = None
    finished: float = None
    state: object = None
    counts: list = field(default_factory=list)
    bytes: int = 0
    remaining: int = 0         # steps of the budget not yet issued to the group

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class Server:
    """Continuous batching of simulations on one GPU."""

    def __init__(self, budget_bytes: float = 160e9, burst_steps: int = 16, max_live: int = 4096,
                 keep_state: bool = True, stream=None):
        self.budget = float(budget_bytes)
        self.burst = int(burst_steps)
        self.max_live = int(max_live)
        self.keep_state = keep_state
        self.stream = stream
        self.group = None
        self.live = {}          # Simulation -> Request
        self.in_use = 0
        self.particle_steps = 0
        self.log = []

    def _admit(self, req: Request, now: float):
        params = params_from_setup(req.setup, precision=req.precision,
                                   history_cap=max(64, int(req.steps) + 8))
        if req.init is not None:
            sim = Simulation(params, init=req.init, stream=self.stream)
        else:
            arrays = req.arrays() if callable(req.arrays) else req.arrays
            sim = Simulation(params, arrays, stream=self.stream)
        req.arrays = None
        if self.group is None:
            self.group = Group([sim], stream=self.stream)
        else:
            self.group.add(sim)
        self.group.budget(sim, int(req.steps))
        req.remaining = int(req.steps)
        req.admitted = now
        self.live[sim] = req
        self.in_use += req.bytes

    def _retire(self, sim: Simulation, req: Request, clock):
        if self.keep_state:
            req.state = sim.state()
        req.counts = sim.counts()
        self.group.remove(sim)
        sim.close()
        req.finished = clock()
        self.in_use -= req.bytes
        self.particle_steps += int(req.setup.n) * int(req.steps)
        del self.live[sim]

    def run(self, requests, time_scale: float = 1.0):
        """Serve the requests (sorted by arrival); returns them with latencies."""
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            r.bytes = sim_bytes_required(params_from_setup(r.setup, precision=r.precision,
                                                           history_cap=max(64, int(r.steps) + 8)))
            if r.bytes > self.budget:
                raise ValueError(f"request {r.rid} needs {r.bytes} bytes, above the budget")
        queue = []
        t0 = time.perf_counter()

        def clock():
            return (time.perf_counter() - t0) / time_scale

        idx = 0
        done = []
        while idx < len(pending) or queue or self.live:
            now = clock()
            while idx < len(pending) and pending[idx].arrival <= now:
                queue.append(pending[idx])
                idx += 1
            # admission in arrival order while the budget allows
            while queue and len(self.live) < self.max_live and \
                    self.in_use + queue[0].bytes <= self.budget:
                self._admit(queue.pop(0), clock())
            if not self.live:
                if idx < len(pending):
                    wait = (pending[idx].arrival - clock()) * time_scale
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                continue
            # one burst of group steps, ending when the live request closest to its end
            # has run its budget (members whose budget is spent are skipped on the
            # device; the group's sync leaves every member where its budget says)
            burst = max(1, min(self.burst, min(r.remaining for r in self.live.values())))
            self.group.step(burst)
            self.group.sync()
            for sim, req in list(self.live.items()):
                req.remaining = max(0, req.remaining - burst)
                if req.remaining == 0:
                    left = self.group.steps_left(sim)
                    if left != 0:
                        raise RuntimeError(f"request {req.rid}: {left} steps left on the "
                                           f"device, none on the host")
                    self._retire(sim, req, clock)
                    done.append(req)
        wall = clock()
        if self.group is not None:
            self.group.close()
            self.group = None
        self.log.append({"wall_s": wall, "particle_steps": self.particle_steps})
        return done, wall


def summarize(done, wall_s):
    lat = np.array([r.latency for r in done], dtype=float)
    ps = sum(int(r.setup.n) * int(r.steps) for r in done)
    return {
        "requests": len(done),
        "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_latency_s": float(lat.mean()) if len(lat) else None,
        "particle_steps": ps,
        "wall_s": wall_s,
        "particle_steps_per_s": ps / wall_s if wall_s > 0 else None,
    }
