"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/osmpm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "osmpm.h")).read()
    return sorted(set(re.findall(r"^(?:osmpm_status|const char\*)\s+(osmpm_\w+)\(", src, re.M)))


def test_header_declares_the_entry_points():
    names = _declared()
    for required in ("osmpm_create_domain", "osmpm_step", "osmpm_schwarz_couple",
                     "osmpm_get_particles", "osmpm_last_error"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2605_09097_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2605_09097_gb300 import osmpm
    assert set(_declared()) == set(osmpm.EXPORTED)


def test_last_error_is_callable_without_gpu():
    from paper_2605_09097_gb300 import osmpm
    assert isinstance(osmpm.osmpm_last_error(), str)


def test_invalid_descriptor_is_rejected_without_touching_the_device():
    """Argument validation happens on the host before any CUDA call."""
    from paper_2605_09097_gb300 import osmpm
    from paper_2605_09097_gb300 import workloads as W
    spec = W.block(2, n_cells=(2, 2))
    desc = osmpm.make_desc(spec)
    desc.dim = 4
    p = spec.particles
    arrs = [p.x, p.v, p.B, p.F, p.vol0, p.mass, p.E, p.nu]
    pin = osmpm.osmpm_particles_in(p.n, *(osmpm._dp(a) for a in arrs),
                                   p.flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    h = ctypes.c_void_p()
    st = osmpm._lib.osmpm_create_domain(ctypes.byref(desc), ctypes.byref(pin), None, None,
                                        ctypes.byref(h))
    assert st == osmpm.OSMPM_E_INVALID
    assert "dim" in osmpm.osmpm_last_error()
