"""The C-ABI library builds, loads and exports every entry point of include/kmc.h;
host-side parameter checks reject bad input before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

import paper_1310_3437_gb300 as kmc
from kmc_inputs import equilibrium_setup, piston_setup

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "kmc.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for want in ["sim_create", "sim_step", "sim_sync", "sim_observe", "sim_destroy",
                 "sim_last_error", "sim_bytes_required", "sim_group_create", "sim_group_step",
                 "sim_group_destroy"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(kmc.library_path() if os.path.exists(kmc.library_path()) else kmc.lib()._name)
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    # sizes follow from the field lists in include/kmc.h
    assert C.sizeof(kmc.kmc_params) == 4 + 4 + 24 + 12 + 4 + 8 * 4 + 8 * 2 + 4 * 4 + 8 * 2 + 4 * 4 + 8
    assert C.sizeof(kmc.kmc_step_counts) == 8 + 4 + 4 + 16 + 4 + 4 + 8 + 8 + 4 + 4


def test_bytes_required_scales_with_n():
    a = kmc.sim_bytes_required(kmc.params_from_setup(equilibrium_setup(n=4096)))
    b = kmc.sim_bytes_required(kmc.params_from_setup(equilibrium_setup(n=1 << 20)))
    assert a > 0 and b > 100 * a
    # guarded binary32 keeps a 24-byte mirror per particle
    c = kmc.sim_bytes_required(kmc.params_from_setup(equilibrium_setup(n=1 << 20),
                                                     precision=kmc.KMC_GUARDED_FP32))
    assert c - b == 24 * (1 << 20)
    assert 100 <= b / (1 << 20) <= 400


@pytest.mark.parametrize("field,value", [
    ("n", 0), ("d0", 0.0), ("dt", -1.0), ("max_rounds", 5), ("precision", 7), ("stencil", 3),
    ("profile_bins", 300), ("cell_scale", 0.5), ("flags", 16), ("flags", 3), ("search_kernel", 4),
    ("n", 0x7FFFF001),
])
def test_invalid_parameters_are_rejected_on_the_host(field, value):
    p = kmc.params_from_setup(piston_setup(n=1000))
    setattr(p, field, value)
    assert kmc.sim_bytes_required(p) == 0
    out = C.c_void_p()
    dummy = C.c_void_p(1)
    rc = kmc.lib().sim_create(C.byref(p), dummy, dummy, dummy, dummy, dummy, dummy, None, None,
                              C.byref(out))
    assert rc == kmc.KMC_EINVAL
    assert out.value is None
    assert kmc.sim_last_error(None) != ""


def test_null_arguments_are_rejected():
    p = kmc.params_from_setup(equilibrium_setup(n=10))
    out = C.c_void_p()
    rc = kmc.lib().sim_create(C.byref(p), None, None, None, None, None, None, None, None,
                              C.byref(out))
    assert rc == kmc.KMC_EINVAL
    assert kmc.lib().sim_step(None, 1) == kmc.KMC_EINVAL
    assert kmc.lib().sim_sync(None) == kmc.KMC_EINVAL
    assert kmc.lib().sim_destroy(None) == kmc.KMC_OK


def test_init_descriptor_layout_and_host_checks():
    assert C.sizeof(kmc.kmc_init) == 4 + 4 + 8 + 8 * 3 + 24 + 8
    assert "sim_create_init" in _declared_functions()
    s = equilibrium_setup(n=1000)
    good_blast = {"kind": kmc.KMC_INIT_BLAST, "n_hot": 10, "sigma": 1.0, "sigma_hot": 10.0,
                  "center": (0.5, 0.5, 0.5), "radius": 0.1}
    bad = [
        ({"kind": 0}, 0), ({"kind": 4}, 0), ({"kind": kmc.KMC_INIT_MAXWELL, "sigma": -1.0}, 0),
        ({"kind": kmc.KMC_INIT_MAXWELL, "sigma": float("nan")}, 0),
        ({"kind": kmc.KMC_INIT_EQUAL_SPEED, "speed": float("inf")}, 0),
        (dict(good_blast, n_hot=1001), 0), (dict(good_blast, radius=0.0), 0),
        (dict(good_blast, center=(0.5, 0.5, 0.95)), 0), (dict(good_blast, center=(0.1, 0.5, 0.5)), 0),
        (good_blast, kmc.KMC_FLAG_PLANAR),
    ]
    for spec, flags in bad:
        p = kmc.params_from_setup(s)
        p.flags = flags
        out = C.c_void_p()
        rc = kmc.lib().sim_create_init(C.byref(p), C.byref(kmc.init_from_spec(spec)), None,
                                       C.byref(out))
        assert rc == kmc.KMC_EINVAL, spec
        assert out.value is None
        assert kmc.sim_last_error(None) != ""
    out = C.c_void_p()
    assert kmc.lib().sim_create_init(C.byref(kmc.params_from_setup(s)), None, None,
                                     C.byref(out)) == kmc.KMC_EINVAL


def test_mixture_tables_are_checked_on_the_host():
    import numpy as np
    from kmc_inputs import mixture_setup
    s = mixture_setup(n=100)
    dummy = C.c_void_p(1)
    sp = np.zeros(100, np.uint8)
    for masses, radii, nsp, d0 in [((1.0, 0.0), (0.01, 0.01), 2, 0.1), ((1.0, 2.0), (0.01, -1.0), 2, 0.1),
                                   ((1.0,), (0.01,), 0, 0.1), ((1.0, 2.0), (0.01, 0.06), 2, 0.1),
                                   ((1.0, float("inf")), (0.01, 0.01), 2, 0.1)]:
        p = kmc.params_from_setup(s)
        p.d0 = d0
        m = np.asarray(masses + (1.0,) * 4, np.float64)
        r = np.asarray(radii + (0.01,) * 4, np.float64)
        out = C.c_void_p()
        rc = kmc.lib().sim_create_mixture(C.byref(p), dummy, dummy, dummy, dummy, dummy, dummy,
                                          None, sp.ctypes.data, nsp, m.ctypes.data, r.ctypes.data,
                                          None, C.byref(out))
        assert rc == kmc.KMC_EINVAL, (masses, radii, nsp)
        assert out.value is None


def test_binding_constants_match_the_header():
    """Every integer #define of include/kmc.h has the same value in the binding."""
    text = open(HEADER).read()
    defs = re.findall(r"^#define\s+(KMC_[A-Z0-9_]+)\s+\(?(-?(?:0x[0-9A-Fa-f]+|\d+))u?\)?", text, flags=re.M)
    assert len(defs) > 20
    missing = []
    for name, val in defs:
        want = int(val, 16) if val.lower().startswith("0x") or val.lower().startswith("-0x") else int(val)
        if not hasattr(kmc, name):
            missing.append(name)
            continue
        assert getattr(kmc, name) == want, name
    assert not missing, missing
