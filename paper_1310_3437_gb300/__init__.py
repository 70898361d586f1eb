"""GB300 (sm_103a) kinetic Monte Carlo collision step -- Python binding of libkmc.

The functions here carry the names of the C ABI in ``include/kmc.h`` and only
marshal arguments (ctypes); every step of the method runs in the CUDA kernels of
``libkmc.so``.  PyTorch is used for device memory and streams only.  If the
library cannot be built or loaded, importing the binding raises: there is no CPU
fallback.

The paper is Howell et al., "Parallelization of Kinetic Theory Simulations"
(Sec. 2: binning, closest-approach partner search, mutual choice, collision,
streaming and boundaries).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

KMC_OK = 0
KMC_EINVAL = -1
KMC_ENOMEM = -2
KMC_ECUDA = -3
KMC_ETIMEOUT = -4
KMC_EOVERFLOW = -5
KMC_ESTATE = -6
KMC_ERANDOM = -7

KMC_PERIODIC = 0
KMC_REFLECT = 1
KMC_ABSORB = 2
KMC_FP64 = 0
KMC_GUARDED_FP32 = 1

KMC_OBS_STATE = 1
KMC_OBS_PARTNERS = 2
KMC_OBS_COUNTS = 3
KMC_OBS_PROFILES = 4
KMC_OBS_EDGES = 5
KMC_OBS_STEP = 6
KMC_OBS_LAUNCHES = 7
KMC_OBS_PHASE_MS = 8
KMC_OBS_VMAX = 9
KMC_OBS_DOMAINS = 10

KMC_NONE = 0xFFFFFFFF
KMC_ABSORBED = 0xFFFFFFFE

KMC_FLAG_NO_SPLIT = 1
KMC_FLAG_FORCE_SPLIT = 2
KMC_FLAG_PLANAR = 4
KMC_FLAG_SCAN_WAIT_TEST = 8

KMC_INIT_MAXWELL = 1
KMC_INIT_EQUAL_SPEED = 2
KMC_INIT_BLAST = 3

KMC_SEARCH_AUTO = 0
KMC_SEARCH_PARTICLE = 1
KMC_SEARCH_CELL = 2
KMC_SEARCH_ROW = 3


class kmc_params(C.Structure):
    _fields_ = [
        ("n", C.c_uint32), ("flags", C.c_uint32),
        ("box", C.c_double * 3),
        ("bc", C.c_int32 * 3),
        ("max_rounds", C.c_int32),
        ("piston_x0", C.c_double), ("piston_u", C.c_double),
        ("d0", C.c_double), ("dt", C.c_double),
        ("seed", C.c_uint64), ("step0", C.c_uint64),
        ("precision", C.c_int32), ("profile_bins", C.c_int32),
        ("profile_every", C.c_int32), ("stencil", C.c_int32),
        ("profile_range", C.c_double), ("cell_scale", C.c_double),
        ("edge_cap", C.c_uint32), ("history_cap", C.c_uint32),
        ("profile_cap", C.c_uint32), ("search_kernel", C.c_int32),
        ("split_min_occ", C.c_double),
    ]


class kmc_init(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("pad0", C.c_uint32), ("n_hot", C.c_uint64),
                ("sigma", C.c_double), ("speed", C.c_double), ("sigma_hot", C.c_double),
                ("center", C.c_double * 3), ("radius", C.c_double)]


class kmc_step_counts(C.Structure):
    _fields_ = [
        ("step", C.c_uint64), ("collisions", C.c_uint32), ("edges", C.c_uint32),
        ("round_pairs", C.c_uint32 * 4), ("survivors", C.c_uint32), ("cells", C.c_uint32),
        ("pair_tests", C.c_uint64), ("fast_tests", C.c_uint64),
        ("absorbed", C.c_uint32), ("live", C.c_uint32),
    ]


class KmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libkmc error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

_P = C.c_void_p


def lib():
    """Load libkmc.so (building it from source if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            L.sim_create.argtypes = [C.POINTER(kmc_params), _P, _P, _P, _P, _P, _P, _P, _P,
                                     C.POINTER(_P)]
            L.sim_create.restype = C.c_int
            L.sim_create_mixture.argtypes = [C.POINTER(kmc_params), _P, _P, _P, _P, _P, _P, _P,
                                             _P, C.c_uint32, _P, _P, _P, C.POINTER(_P)]
            L.sim_create_mixture.restype = C.c_int
            L.sim_create_init.argtypes = [C.POINTER(kmc_params), C.POINTER(kmc_init), _P,
                                          C.POINTER(_P)]
            L.sim_create_init.restype = C.c_int
            L.sim_create_domains.argtypes = [C.POINTER(kmc_params), C.c_uint32, _P, _P, _P, _P,
                                             _P, _P, _P, _P, C.POINTER(_P)]
            L.sim_create_domains.restype = C.c_int
            L.sim_step.argtypes = [_P, C.c_uint32]
            L.sim_step.restype = C.c_int
            L.sim_sync.argtypes = [_P]
            L.sim_sync.restype = C.c_int
            L.sim_observe.argtypes = [_P, C.c_int, _P, C.c_size_t]
            L.sim_observe.restype = C.c_int64
            L.sim_set_timing.argtypes = [_P, C.c_int]
            L.sim_set_timing.restype = C.c_int
            L.sim_destroy.argtypes = [_P]
            L.sim_destroy.restype = C.c_int
            L.sim_last_error.argtypes = [_P]
            L.sim_last_error.restype = C.c_char_p
            L.sim_bytes_required.argtypes = [C.POINTER(kmc_params)]
            L.sim_bytes_required.restype = C.c_size_t
            L.sim_group_create.argtypes = [C.POINTER(_P), C.c_uint32, _P, C.POINTER(_P)]
            L.sim_group_create.restype = C.c_int
            L.sim_group_add.argtypes = [_P, _P]
            L.sim_group_add.restype = C.c_int
            L.sim_group_remove.argtypes = [_P, _P]
            L.sim_group_remove.restype = C.c_int
            L.sim_group_budget.argtypes = [_P, _P, C.c_uint32]
            L.sim_group_budget.restype = C.c_int
            L.sim_group_step.argtypes = [_P, C.c_uint32]
            L.sim_group_step.restype = C.c_int
            L.sim_group_steps_left.argtypes = [_P, _P]
            L.sim_group_steps_left.restype = C.c_int64
            L.sim_group_sync.argtypes = [_P]
            L.sim_group_sync.restype = C.c_int
            L.sim_group_destroy.argtypes = [_P]
            L.sim_group_destroy.restype = C.c_int
            L.sim_profile_static.argtypes = [_P, _P, _P, _P, C.c_uint32, C.c_int32, C.c_double,
                                             _P, _P]
            L.sim_profile_static.restype = C.c_int
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _check(rc, handle=None):
    if rc < 0:
        msg = lib().sim_last_error(handle)
        raise KmcError(int(rc), msg.decode() if msg else "")
    return rc


# ---- thin wrappers with the C names ------------------------------------------ #
def sim_create(params: kmc_params, x, y, z, vx, vy, vz, last=None, stream=None):
    out = _P()
    rc = lib().sim_create(C.byref(params), x, y, z, vx, vy, vz, last, stream, C.byref(out))
    _check(rc, None)
    return out.value


def sim_create_mixture(params: kmc_params, x, y, z, vx, vy, vz, last, species, nspecies: int,
                       mass, radius, stream=None):
    out = _P()
    rc = lib().sim_create_mixture(C.byref(params), x, y, z, vx, vy, vz, last, species,
                                  int(nspecies), mass, radius, stream, C.byref(out))
    _check(rc, None)
    return out.value


def sim_create_init(params: kmc_params, init: kmc_init, stream=None):
    out = _P()
    rc = lib().sim_create_init(C.byref(params), C.byref(init), stream, C.byref(out))
    _check(rc, None)
    return out.value


def sim_create_domains(params: kmc_params, ndomains: int, x, y, z, vx, vy, vz, last=None,
                       stream=None):
    out = _P()
    rc = lib().sim_create_domains(C.byref(params), int(ndomains), x, y, z, vx, vy, vz, last,
                                  stream, C.byref(out))
    _check(rc, None)
    return out.value


def init_from_spec(spec: dict) -> kmc_init:
    """kmc_init from a dict with the descriptor's field names."""
    d = kmc_init()
    d.kind = int(spec["kind"])
    d.n_hot = int(spec.get("n_hot", 0))
    d.sigma = float(spec.get("sigma", 1.0))
    d.speed = float(spec.get("speed", 1.0))
    d.sigma_hot = float(spec.get("sigma_hot", 1.0))
    for k, c in enumerate(spec.get("center", (0.5, 0.5, 0.5))):
        d.center[k] = float(c)
    d.radius = float(spec.get("radius", 0.0))
    return d


def sim_step(sim, nsteps: int):
    return _check(lib().sim_step(sim, nsteps), sim)


def sim_sync(sim):
    return _check(lib().sim_sync(sim), sim)


def sim_observe(sim, what: int, dst, dst_bytes: int):
    return _check(lib().sim_observe(sim, what, dst, dst_bytes), sim)


def sim_set_timing(sim, enable: bool):
    return _check(lib().sim_set_timing(sim, 1 if enable else 0), sim)


def sim_destroy(sim):
    return lib().sim_destroy(sim)


def sim_last_error(sim=None) -> str:
    m = lib().sim_last_error(sim)
    return m.decode() if m else ""


def sim_bytes_required(params: kmc_params) -> int:
    return int(lib().sim_bytes_required(C.byref(params)))


def sim_group_create(sims, stream=None):
    arr = (_P * len(sims))(*sims)
    out = _P()
    _check(lib().sim_group_create(arr, len(sims), stream, C.byref(out)), None)
    return out.value


def sim_group_add(group, sim):
    return _check(lib().sim_group_add(group, sim), None)


def sim_group_remove(group, sim):
    return _check(lib().sim_group_remove(group, sim), None)


def sim_group_budget(group, sim, nsteps: int):
    return _check(lib().sim_group_budget(group, sim, nsteps), None)


def sim_group_step(group, nsteps: int):
    return _check(lib().sim_group_step(group, nsteps), None)


def sim_group_steps_left(group, sim) -> int:
    return int(_check(lib().sim_group_steps_left(group, sim), None))


def sim_group_sync(group):
    return _check(lib().sim_group_sync(group), None)


def sim_group_destroy(group):
    return lib().sim_group_destroy(group)


def sim_profile_static(x, vx, vy, vz, n: int, bins: int, range_: float, out, stream=None):
    """Allocation-free x-profile of caller-owned device arrays (pointers)."""
    rc = lib().sim_profile_static(x, vx, vy, vz, int(n), int(bins), float(range_), out, stream)
    if rc < 0:
        raise KmcError(int(rc), "sim_profile_static rejected its arguments (see stderr)")
    return rc


from .sim import Simulation, Group, params_from_setup  # noqa: E402,F401
