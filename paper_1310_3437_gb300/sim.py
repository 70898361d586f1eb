"""Object wrappers over the C ABI: a simulation and a group of simulations.

Only argument marshalling happens here.  Arrays may be NumPy (host) or torch CUDA
tensors (device); the library copies with cudaMemcpyDefault either way.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import (KMC_FP64, KMC_GUARDED_FP32, KMC_NONE, KMC_OBS_COUNTS, KMC_OBS_EDGES,
               KMC_OBS_LAUNCHES, KMC_OBS_PARTNERS, KMC_OBS_PHASE_MS, KMC_OBS_PROFILES,
               KMC_OBS_STATE, KMC_OBS_STEP, KMC_OBS_VMAX, KMC_OBS_DOMAINS, kmc_params, sim_set_timing,
               kmc_step_counts, sim_create, sim_create_init, sim_create_mixture, sim_create_domains,
               init_from_spec, sim_destroy, sim_group_add, sim_group_budget,
               sim_group_create, sim_group_destroy, sim_group_remove, sim_group_step,
               sim_group_steps_left, sim_group_sync, sim_observe, sim_step, sim_sync)


def params_from_setup(setup, precision=KMC_FP64, stencil=1, cell_scale=1.0, step0=0,
                      edge_cap=0, history_cap=0, profile_cap=0, search_kernel=0,
                      split_min_occ=0.0, flags=0) -> kmc_params:
    """kmc_params from any object with the fields n, box, bc, piston_x0, piston_u, d0,
    dt, seed, max_rounds, profile_bins, profile_every, profile_range."""
    p = kmc_params()
    p.n = int(setup.n)
    for a in range(3):
        p.box[a] = float(setup.box[a])
        p.bc[a] = int(setup.bc[a])
    p.max_rounds = int(getattr(setup, "max_rounds", 4))
    p.piston_x0 = float(getattr(setup, "piston_x0", 0.0)) or float(setup.box[0])
    p.piston_u = float(getattr(setup, "piston_u", 0.0))
    p.d0 = float(setup.d0)
    p.dt = float(setup.dt)
    p.seed = int(setup.seed)
    p.step0 = int(step0)
    p.precision = int(precision)
    p.profile_bins = int(getattr(setup, "profile_bins", 0))
    p.profile_every = int(getattr(setup, "profile_every", 0))
    p.profile_range = float(getattr(setup, "profile_range", 1.0))
    p.stencil = int(stencil)
    p.cell_scale = float(cell_scale)
    p.edge_cap = int(edge_cap)
    p.history_cap = int(history_cap)
    p.profile_cap = int(profile_cap)
    p.search_kernel = int(search_kernel)
    p.split_min_occ = float(split_min_occ)
    p.flags = int(flags) | (4 if getattr(setup, "planar", False) else 0)  # KMC_FLAG_PLANAR
    return p


def _ptr(a):
    """(pointer, keepalive) of a NumPy array or a torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.data_ptr(), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a)
    return arr.ctypes.data, arr


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return None


class Simulation:
    """One simulation: state on the device, stepped by the library's kernels."""

    def __init__(self, params: kmc_params, arrays=None, last=None, stream=None, init=None,
                 mixture=None, domains=None):
        """From host or device arrays (x, y, z, vx, vy, vz) and optional last partners,
        or, with ``init`` (a dict with kmc_init's fields), from a state drawn on the
        device.  ``mixture``: (species per id, masses, radii) for a mixture.
        ``domains``: decompose into that many x slabs (sim_create_domains)."""
        self.params = params
        self.n = int(params.n)
        self.group = None
        if init is not None:
            if stream is None:
                stream = _torch_stream()
            self._init = init_from_spec(init)
            self.handle = sim_create_init(params, self._init, stream)
            return
        cols = [np.asarray(a, dtype=np.float64) if not hasattr(a, "data_ptr") else a for a in arrays]
        ptrs, self._keep = [], []
        for a in cols:
            p, k = _ptr(a)
            ptrs.append(p)
            self._keep.append(k)
        lp = None
        if last is not None:
            if not hasattr(last, "data_ptr"):
                last = np.ascontiguousarray(last, dtype=np.uint32)
            lp, k = _ptr(last)
            self._keep.append(k)
        if stream is None:
            stream = _torch_stream()
        if domains is not None:
            if mixture is not None:
                raise ValueError("a decomposition of a mixture is not supported")
            self.handle = sim_create_domains(params, int(domains), *ptrs, lp, stream)
        elif mixture is not None:
            sp, ms, rs = mixture
            sp, k1 = _ptr(sp if hasattr(sp, "data_ptr") else np.ascontiguousarray(sp, np.uint8))
            ms = np.ascontiguousarray(ms, dtype=np.float64)
            rs = np.ascontiguousarray(rs, dtype=np.float64)
            self._keep += [k1, ms, rs]
            self.handle = sim_create_mixture(params, *ptrs, lp, sp, len(ms), ms.ctypes.data,
                                             rs.ctypes.data, stream)
        else:
            self.handle = sim_create(params, *ptrs, lp, stream)
        self._keep = None
        self.group = None

    # -- stepping --
    def step(self, nsteps: int = 1):
        sim_step(self.handle, int(nsteps))
        return self

    def sync(self):
        sim_sync(self.handle)
        return self

    # -- observables (host NumPy copies) --
    def state(self):
        """(six float64 arrays x, y, z, vx, vy, vz in id order, uint32 last partner)."""
        n = self.n
        buf = np.empty(n * 52, dtype=np.uint8)
        sim_observe(self.handle, KMC_OBS_STATE, buf.ctypes.data, buf.nbytes)
        f = buf[: 48 * n].view(np.float64).reshape(6, n)
        last = buf[48 * n:].view(np.uint32)
        return [f[i].copy() for i in range(6)], last.copy()

    def state_device(self, out):
        """Gather the state into a device buffer (torch uint8 tensor of 52 n bytes)."""
        return sim_observe(self.handle, KMC_OBS_STATE, out.data_ptr(), out.numel() * out.element_size())

    def partners(self):
        out = np.empty(self.n, dtype=np.uint32)
        sim_observe(self.handle, KMC_OBS_PARTNERS, out.ctypes.data, out.nbytes)
        return out

    def edges(self, cap=None):
        cap = cap or max(1024, self.n)
        while True:
            out = np.empty((cap, 2), dtype=np.uint32)
            try:
                cnt = sim_observe(self.handle, KMC_OBS_EDGES, out.ctypes.data, out.nbytes)
            except Exception:
                cap *= 4
                if cap > 64 * self.n + 65536:
                    raise
                continue
            e = out[:cnt]
            order = np.lexsort((e[:, 1], e[:, 0]))
            return e[order]

    def counts(self):
        cap = max(1, int(self.params.history_cap or 4096))
        arr = (kmc_step_counts * cap)()
        cnt = sim_observe(self.handle, KMC_OBS_COUNTS, C.addressof(arr), C.sizeof(arr))
        return [{"step": int(r.step), "collisions": int(r.collisions), "edges": int(r.edges),
                 "round_pairs": [int(x) for x in r.round_pairs], "survivors": int(r.survivors),
                 "cells": int(r.cells), "pair_tests": int(r.pair_tests),
                 "fast_tests": int(r.fast_tests), "absorbed": int(r.absorbed),
                 "live": int(r.live)} for r in arr[:cnt]]

    def profiles(self):
        bins = int(self.params.profile_bins)
        if bins <= 0:
            return np.zeros((0, 0, 7))
        cap = int(self.params.profile_cap or 64)
        out = np.empty((cap, bins, 7))
        cnt = sim_observe(self.handle, KMC_OBS_PROFILES, out.ctypes.data, out.nbytes)
        return out[:cnt].copy()

    def launches(self) -> int:
        out = np.zeros(1, dtype=np.uint64)
        sim_observe(self.handle, KMC_OBS_LAUNCHES, out.ctypes.data, out.nbytes)
        return int(out[0])

    def set_timing(self, enable: bool):
        sim_set_timing(self.handle, enable)

    def phase_ms(self):
        """Accumulated ms of the sort, search, matching and push phases, the number of
        steps timed (after set_timing(True)), and the ms of the slow-population search
        kernels alone (part of the search phase)."""
        out = np.zeros(6)
        sim_observe(self.handle, KMC_OBS_PHASE_MS, out.ctypes.data, out.nbytes)
        return {"sort": out[0], "search": out[1], "match": out[2], "push": out[3],
                "steps": int(out[4]), "search_slow": out[5]}

    def vmax(self) -> float:
        """Largest particle speed of the current state (binary64, correctly rounded)."""
        out = np.zeros(1)
        sim_observe(self.handle, KMC_OBS_VMAX, out.ctypes.data, out.nbytes)
        return float(out[0])

    def domains(self):
        """(owned, ghosts) per domain in the last step of a decomposition."""
        cap = 2 * 64
        out = np.zeros(cap, dtype=np.uint32)
        cnt = sim_observe(self.handle, KMC_OBS_DOMAINS, out.ctypes.data, out.nbytes)
        return out[: cnt // 2].copy(), out[cnt // 2: cnt].copy()

    def step_index(self) -> int:
        out = np.zeros(1, dtype=np.uint64)
        sim_observe(self.handle, KMC_OBS_STEP, out.ctypes.data, out.nbytes)
        return int(out[0])

    def close(self):
        if getattr(self, "handle", None):
            sim_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Simulations stepped together: one launch per kernel for all members."""

    def __init__(self, sims, stream=None):
        if stream is None:
            stream = _torch_stream()
        self.members = list(sims)
        self.handle = sim_group_create([s.handle for s in sims], stream)
        for s in sims:
            s.group = self

    def add(self, sim):
        sim_group_add(self.handle, sim.handle)
        self.members.append(sim)
        sim.group = self

    def remove(self, sim):
        sim_group_remove(self.handle, sim.handle)
        self.members.remove(sim)
        sim.group = None

    def budget(self, sim, nsteps: int):
        sim_group_budget(self.handle, sim.handle, int(nsteps))

    def step(self, nsteps: int = 1):
        sim_group_step(self.handle, int(nsteps))

    def steps_left(self, sim) -> int:
        return sim_group_steps_left(self.handle, sim.handle)

    def sync(self):
        sim_group_sync(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            for s in self.members:
                s.group = None
            sim_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Simulation", "Group", "params_from_setup", "KMC_FP64", "KMC_GUARDED_FP32", "KMC_NONE"]
