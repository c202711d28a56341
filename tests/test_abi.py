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


def _create(desc_edit=None, part_edit=None):
    from paper_2605_09097_gb300 import osmpm
    from paper_2605_09097_gb300 import workloads as W
    spec = W.block(2, n_cells=(2, 2))
    desc = osmpm.make_desc(spec)
    if desc_edit:
        desc_edit(desc)
    p = spec.particles
    arrs = [a.copy() for a in (p.x, p.v, p.B, p.F, p.vol0, p.mass, p.E, p.nu)]
    if part_edit:
        part_edit(arrs)
    pin = osmpm.osmpm_particles_in(p.n, *(osmpm._dp(a) for a in arrs),
                                   p.flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    h = ctypes.c_void_p()
    st = osmpm._lib.osmpm_create_domain(ctypes.byref(desc), ctypes.byref(pin), None, None,
                                        ctypes.byref(h))
    return st, osmpm.osmpm_last_error(), h


def _set(field, value):
    def edit(d):
        setattr(d, field, value)
    return edit


def _res0(d):
    d.res[0] = 3


def _reserved(d):
    d.reserved[1] = 7


@pytest.mark.parametrize("edit,word", [
    (_set("precision", 2), "precision"),
    (_set("pcg_mode", 3), "pcg_mode"),
    (_set("launch_mode", 2), "launch_mode"),
    (_set("hvp_mode", 3), "hvp_mode"),
    (_set("cg_eta_max", 1.0), "cg_eta_max"),
    (_set("dx", 0.0), "dx"),
    (_set("newton_max", 0), "solver controls"),
    (_res0, "res[0]"),
    (_reserved, "reserved"),
])
def test_descriptor_checks_run_on_the_host(edit, word):
    from paper_2605_09097_gb300 import osmpm
    st, msg, h = _create(desc_edit=edit)
    assert st == osmpm.OSMPM_E_INVALID and word in msg and not h.value


def _nu_half(a):
    a[7][0] = 0.5


def _x_nan(a):
    a[0][1, 0] = float("nan")


@pytest.mark.parametrize("edit,status,word", [
    (_nu_half, "OSMPM_E_INVALID", "nu"),
    (_x_nan, "OSMPM_E_NONFINITE", "non-finite"),
])
def test_particle_checks_run_on_the_host(edit, status, word):
    from paper_2605_09097_gb300 import osmpm
    st, msg, h = _create(part_edit=edit)
    assert st == getattr(osmpm, status) and word in msg and not h.value


def test_batch_and_stream_argument_checks_run_on_the_host():
    from paper_2605_09097_gb300 import osmpm
    lib = osmpm._lib
    assert lib.osmpm_create_stream(None) == osmpm.OSMPM_E_INVALID
    assert lib.osmpm_destroy_stream(None) == osmpm.OSMPM_OK
    # bad candidate lists are refused before any pair is touched
    fake = (ctypes.c_void_p * 1)(ctypes.c_void_p(1))
    sd = (osmpm.osmpm_schwarz_desc * 1)()
    best = ctypes.c_int32(-1)
    for cands in ([], [8, 0]):
        arr = (ctypes.c_int32 * max(len(cands), 1))(*cands)
        st = lib.osmpm_autotune_batch(fake, fake, 1, 0.01, sd, arr, len(cands), ctypes.byref(best), None)
        assert st == osmpm.OSMPM_E_INVALID and best.value == -1
    st = lib.osmpm_schwarz_couple_batch(None, None, 1, 0.01, None, 1, None, None)
    assert st == osmpm.OSMPM_E_INVALID
    c = osmpm.osmpm_counters()
    assert lib.osmpm_get_counters(None, ctypes.byref(c)) == osmpm.OSMPM_OK and c.launches >= 0


def test_no_cpu_fallback_without_a_gpu():
    """On a host without a CUDA device the product path fails loudly: a
    valid domain cannot be created (the library's first device allocation
    fails), and nothing falls back to a CPU computation."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2605_09097_gb300 import osmpm
    from paper_2605_09097_gb300 import workloads as W
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.Domain(W.cantilever(), stream=0, use_torch_allocator=False)
    assert e.value.status in (osmpm.OSMPM_E_CUDA, osmpm.OSMPM_E_NOMEM)
