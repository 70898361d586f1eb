"""Exchange schedule of the domain decomposition across processes (Sec. 4,
"Hybrid Simulations"): one process per x slab, the paper's four communication
phases as point-to-point messages of ``torch.distributed``.

  1. ghosts: each process counts the particles it owns within the reach R of every
     other slab, sends the counts first, then the particles (id, state, last
     partner) -- the paper sends the counts so the receiver can size its buffers;
  2. the global v_max: an all-reduce (max) of the largest squared speed, which gives
     the common reach R = d0 + 2 v_max dt (the paper syncs its adaptive time step);
  3. collision partners: per matching round, the choice (global id) of every owned
     particle that is a ghost elsewhere goes to the processes that hold the ghost;
  4. migration: after the push, the particles whose x left the slab go to the process
     that owns their new position.

On one GPU, ``sim_create_domains`` runs the same four phases between the domains of
one batch through id-indexed device buffers; this module is the host-side schedule
for one process per domain (with the gloo backend, across CPU processes), and it
shares the slab bounds, the ownership rule and the ghost criterion with it.
"""
from __future__ import annotations

import math

import numpy as np

# one row per particle: id, x, y, z, vx, vy, vz, last partner (ids < 2^53 are exact)
ROW = 8
NONE = 0xFFFFFFFF


def slab_bounds(xmax: float, ndomains: int) -> np.ndarray:
    """X_k = xmax k / P: domain k owns X_k <= x < X_(k+1) (the last one all above)."""
    return np.array([xmax * float(k) / float(ndomains) for k in range(ndomains + 1)])


def owner_of(x, X) -> np.ndarray:
    """Largest k with X_k <= x, clamped to [0, P - 1]."""
    P = len(X) - 1
    k = np.searchsorted(X, np.asarray(x, dtype=np.float64), side="right") - 1
    return np.clip(k, 0, P - 1)


def slab_distance(x, X, k: int, periodic: bool, Lx: float) -> np.ndarray:
    """Distance along x from x to slab k (the shorter way round on a periodic axis)."""
    x = np.asarray(x, dtype=np.float64)
    a, b = X[k], X[k + 1]
    d = np.where(x < a, a - x, np.where(x >= b, x - b, 0.0))
    if periodic:
        w = np.where(x < a, (x - b) + Lx, np.where(x >= b, (a - x) + Lx, 0.0))
        d = np.where((d > 0.0) & (w < d), w, d)
    return d


def reach(vmax2: float, d0: float, dt: float) -> float:
    """Ghost reach d0 + 2 v_max dt, widened by a relative 2^-20 (an extra ghost changes
    no result, a missing one would)."""
    r = d0 + 2.0 * math.sqrt(vmax2) * dt
    return r * (1.0 + 2.0 ** -20) + 2.0 ** -1000


class DomainRank:
    """The particles one process owns, and its side of the four phases."""

    def __init__(self, rank: int, world: int, X, rows: np.ndarray, periodic: bool, Lx: float,
                 d0: float, dt: float):
        self.rank, self.world = rank, world
        self.X = np.asarray(X, dtype=np.float64)
        self.rows = np.ascontiguousarray(rows, dtype=np.float64).reshape(-1, ROW)
        self.periodic, self.Lx, self.d0, self.dt = periodic, Lx, d0, dt
        self.ghosts = np.zeros((0, ROW))
        self.sent_ghost_ids = {}   # destination -> ids of owned particles it holds as ghosts
        self.counts_sent = {}
        self.counts_received = {}

    # -- message passing: counts first, then the rows --------------------------
    def _exchange(self, payload: dict) -> dict:
        import torch
        import torch.distributed as dist

        others = [r for r in range(self.world) if r != self.rank]
        cout = {d: torch.tensor([len(payload.get(d, ()))], dtype=torch.int64) for d in others}
        cin = {s: torch.zeros(1, dtype=torch.int64) for s in others}
        reqs = [dist.isend(cout[d], d) for d in others] + [dist.irecv(cin[s], s) for s in others]
        for q in reqs:
            q.wait()
        got = {s: torch.empty((int(cin[s].item()), ROW), dtype=torch.float64) for s in others}
        reqs = []
        for d in others:
            if int(cout[d].item()):
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(payload[d])), d))
        for s in others:
            if int(cin[s].item()):
                reqs.append(dist.irecv(got[s], s))
        for q in reqs:
            q.wait()
        self.counts_sent = {d: int(cout[d].item()) for d in others}
        self.counts_received = {s: int(cin[s].item()) for s in others}
        return {s: got[s].numpy() for s in others}

    # -- phase 2 ----------------------------------------------------------------
    def global_vmax2(self) -> float:
        import torch
        import torch.distributed as dist

        v = self.rows[:, 4:7]
        local = float(((v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2]).max()) \
            if len(v) else 0.0
        t = torch.tensor([local], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # -- phase 1 ----------------------------------------------------------------
    def exchange_ghosts(self, R: float) -> np.ndarray:
        payload = {}
        for d in range(self.world):
            if d == self.rank:
                continue
            near = slab_distance(self.rows[:, 1], self.X, d, self.periodic, self.Lx) < R
            payload[d] = self.rows[near]
            self.sent_ghost_ids[d] = self.rows[near, 0].astype(np.int64)
        got = self._exchange(payload)
        self.ghosts = np.concatenate([got[s] for s in sorted(got)] or [np.zeros((0, ROW))])
        return self.ghosts

    # -- phase 3 ----------------------------------------------------------------
    def exchange_choices(self, choice_of_owned: dict) -> dict:
        """choice_of_owned: id -> global id chosen (or NONE) for every owned particle;
        returns id -> choice for every ghost this process holds."""
        payload = {}
        for d, ids in self.sent_ghost_ids.items():
            rows = np.zeros((len(ids), ROW))
            rows[:, 0] = ids
            rows[:, 1] = [choice_of_owned.get(int(i), NONE) for i in ids]
            payload[d] = rows
        got = self._exchange(payload)
        out = {}
        for rows in got.values():
            for r in rows:
                out[int(r[0])] = int(r[1])
        return out

    # -- phase 4 ----------------------------------------------------------------
    def migrate(self) -> None:
        dest = owner_of(self.rows[:, 1], self.X)
        payload = {d: self.rows[dest == d] for d in range(self.world) if d != self.rank}
        keep = self.rows[dest == self.rank]
        got = self._exchange(payload)
        self.rows = np.concatenate([keep] + [got[s] for s in sorted(got)])
