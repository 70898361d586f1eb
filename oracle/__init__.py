"""CPU FP64 oracle for the kinetic Monte Carlo collision step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``kmc_oracle.c`` (plain C, FP64,
built with ``-ffp-contract=off``) through ctypes and shares no code with the CUDA
library.  See the header of ``kmc_oracle.c`` for which part of the paper each
function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libkmc_oracle.so")
_lock = threading.Lock()
_lib = None

NONE = 0xFFFFFFFF
ABSORBED = 0xFFFFFFFE  # last-partner value of a particle that left through an absorbing wall


class Params(C.Structure):
    _fields_ = [
        ("n", C.c_uint32), ("pad0", C.c_uint32),
        ("box", C.c_double * 3),
        ("bc", C.c_int32 * 3),
        ("max_rounds", C.c_int32),
        ("piston_x0", C.c_double), ("piston_u", C.c_double),
        ("d0", C.c_double), ("dt", C.c_double),
        ("seed", C.c_uint64),
        ("profile_bins", C.c_int32), ("profile_every", C.c_int32),
        ("profile_range", C.c_double),
        ("search", C.c_int32), ("threads", C.c_int32),
        ("planar", C.c_int32), ("nspecies", C.c_int32),
        ("species", C.POINTER(C.c_uint8)), ("mass", C.POINTER(C.c_double)),
        ("radius", C.POINTER(C.c_double)),
    ]


class Init(C.Structure):
    """Initial-state descriptor of the Philox initialisation (``or_init``)."""
    _fields_ = [("kind", C.c_int32), ("pad0", C.c_int32), ("n_hot", C.c_uint64),
                ("sigma", C.c_double), ("speed", C.c_double), ("sigma_hot", C.c_double),
                ("center", C.c_double * 3), ("radius", C.c_double)]


class Counts(C.Structure):
    _fields_ = [("step", C.c_uint64), ("collisions", C.c_uint32), ("edges", C.c_uint32),
                ("round_pairs", C.c_uint32 * 4), ("absorbed", C.c_uint32), ("live", C.c_uint32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            up = C.POINTER(C.c_uint32)
            L.or_philox4x32_10.argtypes = [up, up, up]
            L.or_unit_vector.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, dp]
            L.or_unit_vector.restype = C.c_int
            L.or_circle_vector.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, dp]
            L.or_circle_vector.restype = C.c_int
            L.or_pair.argtypes = [C.POINTER(Params), C.POINTER(dp), up, C.c_uint32, C.c_uint32,
                                  dp, dp]
            L.or_pair.restype = C.c_int
            L.or_candidate_pairs.argtypes = [C.POINTER(Params), C.POINTER(dp), up, up, up, dp, dp,
                                             C.c_int64]
            L.or_candidate_pairs.restype = C.c_int64
            L.or_step.argtypes = [C.POINTER(Params), C.POINTER(dp), up, C.c_uint64,
                                  C.POINTER(Counts), up, dp, C.POINTER(C.c_int)]
            L.or_step.restype = C.c_int
            L.or_run.argtypes = [C.POINTER(Params), C.POINTER(dp), up, C.c_uint64, C.c_uint32,
                                 C.POINTER(Counts), dp]
            L.or_run.restype = C.c_int
            L.or_vmax2.argtypes = [C.c_uint32, dp, dp, dp]
            L.or_vmax2.restype = C.c_double
            L.or_max_threads.restype = C.c_int
            L.or_log.argtypes = [C.c_double]
            L.or_log.restype = C.c_double
            L.or_log_many.argtypes = [dp, dp, C.c_int64]
            L.or_init_particles.argtypes = [C.POINTER(Init), C.POINTER(Params), up, C.c_int64,
                                            C.POINTER(dp)]
            L.or_init_particles.restype = C.c_int64
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _up(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def params_from(setup, search: int = 1, threads: int = 0) -> Params:
    p = Params()
    p.n = setup.n
    for k in range(3):
        p.box[k] = float(setup.box[k])
        p.bc[k] = int(setup.bc[k])
    p.max_rounds = int(setup.max_rounds)
    p.piston_x0 = float(setup.piston_x0)
    p.piston_u = float(setup.piston_u)
    p.d0 = float(setup.d0)
    p.dt = float(setup.dt)
    p.seed = int(setup.seed)
    p.profile_bins = int(setup.profile_bins)
    p.profile_every = int(setup.profile_every)
    p.profile_range = float(setup.profile_range)
    p.search = int(search)
    p.threads = int(threads)
    p.planar = 1 if getattr(setup, "planar", False) else 0
    sp = getattr(setup, "species", None)
    if sp is not None:
        # mixture: keep the arrays alive with the struct
        p._keep = (np.ascontiguousarray(sp, dtype=np.uint8),
                   np.ascontiguousarray(setup.masses, dtype=np.float64),
                   np.ascontiguousarray(setup.radii, dtype=np.float64))
        p.nspecies = len(p._keep[1])
        p.species = p._keep[0].ctypes.data_as(C.POINTER(C.c_uint8))
        p.mass = _dp(p._keep[1])
        p.radius = _dp(p._keep[2])
    return p


class State:
    """Particle state in id order: six float64 arrays plus last partner (uint32)."""

    def __init__(self, arrays, last=None):
        self.a = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)).copy() for x in arrays]
        n = self.a[0].shape[0]
        self.last = (np.full(n, NONE, dtype=np.uint32) if last is None
                     else np.ascontiguousarray(last, dtype=np.uint32).copy())
        self._ptrs = (C.POINTER(C.c_double) * 6)(*[_dp(x) for x in self.a])

    @property
    def n(self):
        return self.a[0].shape[0]

    def copy(self):
        return State(self.a, self.last)


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_up(c), _up(k), _up(out))
    return out


def log(s):
    """The oracle's own natural logarithm (+, -, *, / only) of an array or scalar."""
    a = np.ascontiguousarray(np.atleast_1d(np.asarray(s, dtype=np.float64)))
    out = np.empty_like(a)
    lib().or_log_many(_dp(a), _dp(out), a.shape[0])
    return out if np.ndim(s) else float(out[0])


def init_struct(spec: dict) -> Init:
    d = Init()
    d.kind = int(spec["kind"])
    d.n_hot = int(spec.get("n_hot", 0))
    d.sigma = float(spec.get("sigma", 1.0))
    d.speed = float(spec.get("speed", 1.0))
    d.sigma_hot = float(spec.get("sigma_hot", 1.0))
    for k, c in enumerate(spec.get("center", (0.5, 0.5, 0.5))):
        d.center[k] = float(c)
    d.radius = float(spec.get("radius", 0.0))
    return d


def init_particles(setup, spec: dict, ids=None):
    """Initial state of the Philox initialisation: six float64 arrays for ``ids``
    (all particles of ``setup`` if None)."""
    ids = (np.arange(setup.n, dtype=np.uint32) if ids is None
           else np.ascontiguousarray(ids, dtype=np.uint32))
    out = [np.zeros(ids.shape[0]) for _ in range(6)]
    ptrs = (C.POINTER(C.c_double) * 6)(*[_dp(x) for x in out])
    d = init_struct(spec)
    p = params_from(setup)
    fails = lib().or_init_particles(C.byref(d), C.byref(p), _up(ids), ids.shape[0], ptrs)
    if fails:
        raise RuntimeError(f"{fails} particle(s) ran out of rejection attempts")
    return out


def unit_vector(seed: int, step: int, pid: int):
    out = np.zeros(3)
    tries = lib().or_unit_vector(seed, step, pid, _dp(out))
    return out, tries


def circle_vector(seed: int, step: int, pid: int):
    """Scatter direction of the planar mode (unit vector in the x-y plane)."""
    out = np.zeros(3)
    tries = lib().or_circle_vector(seed, step, pid, _dp(out))
    return out, tries


def pair(setup, state: State, i: int, j: int, use_last: bool = True):
    p = params_from(setup)
    d2 = C.c_double()
    t = C.c_double()
    ok = lib().or_pair(C.byref(p), state._ptrs, _up(state.last) if use_last else None, i, j,
                       C.byref(d2), C.byref(t))
    return bool(ok), d2.value, t.value


def candidate_pairs(setup, state: State, search: int = 1, threads: int = 0):
    """All unordered candidate pairs (i < j) with their FP64 keys, sorted by (i, j)."""
    p = params_from(setup, search, threads)
    cap = max(16, state.n)
    while True:
        pi = np.zeros(cap, np.uint32)
        pj = np.zeros(cap, np.uint32)
        d2 = np.zeros(cap)
        t = np.zeros(cap)
        cnt = lib().or_candidate_pairs(C.byref(p), state._ptrs, _up(state.last), _up(pi),
                                       _up(pj), _dp(d2), _dp(t), cap)
        if cnt == -(2 ** 63):
            raise MemoryError("oracle allocation failed")
        if cnt >= 0:
            return pi[:cnt], pj[:cnt], d2[:cnt], t[:cnt]
        cap = -cnt


def step(setup, state: State, step_index: int, search: int = 1, threads: int = 0):
    """One step in place; returns (counts dict, partner array, profile or None)."""
    p = params_from(setup, search, threads)
    cnt = Counts()
    partner = np.zeros(state.n, np.uint32)
    prof = np.zeros(max(1, setup.profile_bins) * 7)
    profiled = C.c_int(0)
    rc = lib().or_step(C.byref(p), state._ptrs, _up(state.last), step_index, C.byref(cnt),
                       _up(partner), _dp(prof), C.byref(profiled))
    if rc:
        raise RuntimeError(f"oracle step failed ({rc})")
    counts = counts_dict(cnt)
    return counts, partner, (prof.reshape(-1, 7).copy() if profiled.value else None)


def counts_dict(c: Counts):
    return {"step": int(c.step), "collisions": int(c.collisions), "edges": int(c.edges),
            "round_pairs": [int(x) for x in c.round_pairs], "absorbed": int(c.absorbed),
            "live": int(c.live)}


def run(setup, state: State, step0: int, nsteps: int, search: int = 1, threads: int = 0):
    """nsteps steps in place; returns (list of counts dicts, profiles array [k, bins, 7])."""
    p = params_from(setup, search, threads)
    cnts = (Counts * max(1, nsteps))()
    nprof = 0
    if setup.profile_every > 0 and setup.profile_bins > 0:
        nprof = sum(1 for s in range(step0, step0 + nsteps)
                    if (s + 1) % setup.profile_every == 0)
    prof = np.zeros(max(1, nprof * setup.profile_bins * 7))
    rc = lib().or_run(C.byref(p), state._ptrs, _up(state.last), step0, nsteps, cnts,
                      _dp(prof) if nprof else None)
    if rc:
        raise RuntimeError(f"oracle run failed ({rc})")
    prof_arr = prof[: nprof * setup.profile_bins * 7].reshape(nprof, setup.profile_bins, 7) \
        if nprof else np.zeros((0, max(1, setup.profile_bins), 7))
    return [counts_dict(cnts[s]) for s in range(nsteps)], prof_arr


def vmax2(state: State) -> float:
    return lib().or_vmax2(state.n, _dp(state.a[3]), _dp(state.a[4]), _dp(state.a[5]))


def max_threads() -> int:
    return lib().or_max_threads()
