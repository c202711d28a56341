"""Thin Python binding of the C ABI in ``include/osmpm.h``.

Argument marshalling only: every step of the method runs in the CUDA
library.  Device memory comes from PyTorch's caching allocator and kernels
run on a PyTorch CUDA stream (the current one unless another is given).
Importing this module loads ``_build/libosmpm.so``; it raises if the library
has not been built, and there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, Structure, c_char_p, c_double, c_int32, c_int64,
                    c_size_t, c_uint8, c_uint32, c_void_p)
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(f"the OS-MPM CUDA library is not built ({LIB_PATH}); run "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)

# status codes
OSMPM_OK = 0
OSMPM_E_INVALID = 1
OSMPM_E_NOMEM = 2
OSMPM_E_CUDA = 3
OSMPM_E_NONFINITE = 4
OSMPM_E_NEWTON_MAXITER = 5
OSMPM_E_LINESEARCH = 6
OSMPM_E_OUT_OF_GRID = 7
OSMPM_E_TIMEOUT = 8
OSMPM_E_UNSUPPORTED = 9
OSMPM_W_SCHWARZ_MAXITER = 100

OSMPM_PI_STEP_AVERAGE = 0
OSMPM_PI_LAST_SUBSTEP = 1

OSMPM_FIELD_MASS = 0
OSMPM_FIELD_VN = 1
OSMPM_FIELD_U = 2
OSMPM_FIELD_BMASS = 3
OSMPM_FIELD_RECEIVER = 4
OSMPM_FIELD_BC = 5
OSMPM_FIELD_PLANE_FORCE = 6
OSMPM_FIELD_PLANE_GAP = 7
OSMPM_FIELD_PLANE_ACTIVE = 8

_ALLOC = CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
_FREE = CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class osmpm_allocator(Structure):
    _fields_ = [("alloc", _ALLOC), ("free", _FREE), ("ctx", c_void_p)]


class osmpm_domain_desc(Structure):
    _fields_ = [("dim", c_int32), ("precision", c_int32), ("origin", c_double * 3),
                ("dx", c_double), ("res", c_int32 * 3), ("gravity", c_double * 3),
                ("newton_tol", c_double), ("newton_max", c_int32), ("cg_rtol", c_double),
                ("cg_max", c_int32), ("ls_max", c_int32), ("mass_eps", c_double),
                ("cg_eta_max", c_double), ("pcg_mode", c_int32), ("launch_mode", c_int32),
                ("hvp_mode", c_int32), ("reserved", c_int32 * 3)]


class osmpm_particles_in(Structure):
    _fields_ = [("n", c_int64), ("x", POINTER(c_double)), ("v", POINTER(c_double)),
                ("B", POINTER(c_double)), ("F", POINTER(c_double)),
                ("vol0", POINTER(c_double)), ("mass", POINTER(c_double)),
                ("E", POINTER(c_double)), ("nu", POINTER(c_double)),
                ("flags", POINTER(c_uint8))]


class osmpm_dirichlet(Structure):
    _fields_ = [("kind", c_int32), ("comp_mask", c_uint32), ("lo", c_double * 3),
                ("hi", c_double * 3), ("vel", c_double * 3), ("center", c_double * 3),
                ("axis", c_double * 3), ("omega", c_double)]


class osmpm_schwarz_desc(Structure):
    _fields_ = [("M", c_int32), ("k_max", c_int32), ("eps_conv", c_double), ("tau_B", c_double),
                ("tau_S", c_double), ("eps_tol", c_double), ("pi_source", c_int32),
                ("reserved", c_int32 * 7)]


class osmpm_stats(Structure):
    _fields_ = [("newton_iters", c_int32), ("cg_iters", c_int32), ("ls_halvings", c_int32),
                ("schwarz_iters", c_int32), ("solves", c_int32), ("converged", c_int32),
                ("r_B", c_double), ("r_S", c_double), ("last_dx_inf", c_double),
                ("contact_sets", c_int32), ("pad", c_int32), ("reserved", c_double * 5)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f not in ("reserved", "pad")}


class osmpm_counters(Structure):
    _fields_ = [("launches", c_int64), ("pcg_launches", c_int64), ("pcg_ms", c_double),
                ("pcg_iters", c_int64), ("particles", c_int64), ("dofs", c_int64),
                ("graph_replays", c_int64), ("graphs", c_int32), ("graph_error", c_int32),
                ("hvp_ms", c_double), ("hvp_launches", c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class osmpm_plane(Structure):
    _fields_ = [("enabled", c_int32), ("max_sets", c_int32), ("level", c_double),
                ("cand_hi", c_double), ("spacing", c_double)]


class osmpm_multi_desc(Structure):
    _fields_ = [("n_threads", c_int32), ("dof_tile", c_int32), ("chunk", c_int32),
                ("slot_tiles", c_int32)]


class osmpm_multi_stats(Structure):
    _fields_ = [("batches", c_int64), ("instances", c_int64), ("chunks", c_int64),
                ("max_batch", c_int64), ("particles", c_int64), ("dofs", c_int64),
                ("iterations", c_int64), ("particle_iterations", c_int64),
                ("dof_iterations", c_int64), ("device_ms", c_double), ("hvp_ms", c_double),
                ("hvp_launches", c_int64), ("hvp_particle_iterations", c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class osmpm_noalloc_grid(Structure):
    _fields_ = [("dim", c_int32), ("origin", c_double * 3), ("dx", c_double),
                ("res", c_int32 * 3), ("mass_eps", c_double), ("gravity", c_double * 3),
                ("m", c_void_p), ("vn", c_void_p), ("u", c_void_p), ("s", c_void_p)]


class osmpm_noalloc_particles(Structure):
    _fields_ = [("n", c_int64), ("x", c_void_p), ("F", c_void_p), ("vol0", c_void_p),
                ("mu", c_void_p), ("lam", c_void_p)]


class osmpm_adjoint_out(Structure):
    _fields_ = [("dJ_dE", c_void_p), ("dJ_dx0", c_void_p), ("dJ_dv0", c_void_p),
                ("dJ_dB0", c_void_p), ("dJ_dF0", c_void_p)]


_DP = POINTER(c_double)
_sig = {
    "osmpm_create_domain": (c_int32, [POINTER(osmpm_domain_desc), POINTER(osmpm_particles_in),
                                      POINTER(osmpm_allocator), c_void_p, POINTER(c_void_p)]),
    "osmpm_destroy_domain": (c_int32, [c_void_p]),
    "osmpm_set_dirichlet": (c_int32, [c_void_p, POINTER(osmpm_dirichlet), c_int32]),
    "osmpm_step": (c_int32, [c_void_p, c_double, POINTER(osmpm_stats)]),
    "osmpm_schwarz_couple": (c_int32, [c_void_p, c_void_p, c_double, POINTER(osmpm_schwarz_desc),
                                       POINTER(osmpm_stats)]),
    "osmpm_schwarz_couple_batch": (c_int32, [POINTER(c_void_p), POINTER(c_void_p), c_int32, c_double,
                                             POINTER(osmpm_schwarz_desc), c_int32,
                                             POINTER(osmpm_stats), POINTER(c_int32)]),
    "osmpm_create_stream": (c_int32, [POINTER(c_void_p)]),
    "osmpm_destroy_stream": (c_int32, [c_void_p]),
    "osmpm_autotune_batch": (c_int32, [POINTER(c_void_p), POINTER(c_void_p), c_int32, c_double,
                                       POINTER(osmpm_schwarz_desc), POINTER(c_int32), c_int32,
                                       POINTER(c_int32), _DP]),
    "osmpm_get_info": (c_int32, [c_void_p, POINTER(c_int64), POINTER(c_int32)]),
    "osmpm_get_particles": (c_int32, [c_void_p, _DP, _DP, _DP, _DP]),
    "osmpm_set_particles": (c_int32, [c_void_p, _DP, _DP, _DP, _DP]),
    "osmpm_get_order": (c_int32, [c_void_p, POINTER(c_uint32)]),
    "osmpm_get_grid": (c_int32, [c_void_p, c_int32, _DP]),
    "osmpm_probe_gradient": (c_int32, [c_void_p, c_double, _DP, _DP]),
    "osmpm_probe_hvp": (c_int32, [c_void_p, c_double, _DP, _DP, _DP]),
    "osmpm_probe_energy_change": (c_int32, [c_void_p, c_double, _DP, _DP, c_double, _DP]),
    "osmpm_set_profiling": (c_int32, [c_void_p, c_int32]),
    "osmpm_get_counters": (c_int32, [c_void_p, POINTER(osmpm_counters)]),
    "osmpm_check_wait_timeout": (c_int32, [c_void_p]),
    "osmpm_record": (c_int32, [c_void_p, c_int32]),
    "osmpm_set_plane": (c_int32, [c_void_p, POINTER(osmpm_plane)]),
    "osmpm_autotune_multi": (c_int32, [c_void_p, c_void_p, c_int32, c_double, c_void_p,
                                       POINTER(osmpm_multi_desc), c_int32, POINTER(c_int32),
                                       POINTER(c_double)]),
    "osmpm_schwarz_couple_multi": (c_int32, [c_void_p, c_void_p, c_int32, c_double, c_void_p,
                                             POINTER(osmpm_multi_desc), c_void_p, c_void_p,
                                             POINTER(osmpm_multi_stats)]),
    "osmpm_adjoint": (c_int32, [c_void_p, c_void_p, c_void_p, POINTER(osmpm_adjoint_out),
                                POINTER(osmpm_stats)]),
    "osmpm_energy_change_noalloc": (c_int32, [POINTER(osmpm_noalloc_grid),
                                              POINTER(osmpm_noalloc_particles), c_double,
                                              c_double, c_void_p, c_void_p]),
    "osmpm_last_error": (c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class OsmpmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.osmpm_last_error().decode()
        super().__init__(f"{where}: status {status}: {msg}")


def _check(status: int, where: str, warn_ok: bool = False) -> int:
    if status == OSMPM_OK or (warn_ok and status == OSMPM_W_SCHWARZ_MAXITER):
        return status
    raise OsmpmError(status, where)


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def osmpm_last_error() -> str:
    return _lib.osmpm_last_error().decode()


# ----------------------------------------------------------------------------
# device memory and streams from PyTorch
# ----------------------------------------------------------------------------
def torch_allocator(device: int = 0):
    """An osmpm_allocator backed by torch.cuda's caching allocator."""
    import torch

    def _a(size, ctx, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), device, int(stream or 0))
        except Exception:  # the C side reports OSMPM_E_NOMEM
            return None

    def _f(ptr, size, ctx, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    cb_a, cb_f = _ALLOC(_a), _FREE(_f)
    return osmpm_allocator(cb_a, cb_f, None), (cb_a, cb_f)


def current_stream() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


# ----------------------------------------------------------------------------
# marshalling of the workload descriptions
# ----------------------------------------------------------------------------
def make_desc(spec) -> osmpm_domain_desc:
    g = spec.grid
    d = osmpm_domain_desc()
    d.dim = g.dim
    d.precision = getattr(spec, "precision", 0)
    for a in range(3):
        d.origin[a] = g.origin[a] if a < g.dim else 0.0
        d.res[a] = g.res[a] if a < g.dim else 1
        d.gravity[a] = spec.gravity[a] if a < g.dim else 0.0
    d.dx = g.dx
    d.newton_tol = spec.newton_tol
    d.newton_max = spec.newton_max
    d.cg_rtol = spec.cg_rtol
    d.cg_max = spec.cg_max
    d.ls_max = spec.ls_max
    d.mass_eps = spec.mass_eps
    d.cg_eta_max = getattr(spec, "cg_eta_max", 0.0)
    d.pcg_mode = getattr(spec, "pcg_mode", 0)
    d.launch_mode = getattr(spec, "launch_mode", 0)
    d.hvp_mode = getattr(spec, "hvp_mode", 0)
    return d


def make_rules(rules) -> "ctypes.Array":
    arr = (osmpm_dirichlet * max(1, len(rules)))()
    for i, r in enumerate(rules):
        t = arr[i]
        t.kind = r.kind
        t.comp_mask = r.comp_mask
        for a in range(3):
            t.lo[a] = r.lo[a] if a < len(r.lo) else -1e30
            t.hi[a] = r.hi[a] if a < len(r.hi) else 1e30
            t.vel[a] = r.vel[a] if a < len(r.vel) else 0.0
            t.center[a] = r.center[a] if a < len(r.center) else 0.0
            t.axis[a] = r.axis[a] if a < len(r.axis) else 0.0
        t.omega = r.omega
    return arr


def make_schwarz_desc(sch) -> osmpm_schwarz_desc:
    s = osmpm_schwarz_desc()
    s.M = sch.M
    s.k_max = sch.k_max
    s.eps_conv = sch.eps_conv
    s.tau_B = sch.tau_B
    s.tau_S = sch.tau_S
    s.eps_tol = sch.eps_tol
    s.pi_source = sch.pi_source
    return s


class Domain:
    """Owns one osmpm_domain handle (and the callbacks its allocator needs)."""

    def __init__(self, spec, stream: Optional[int] = None, use_torch_allocator: bool = True,
                 device: int = 0):
        p = spec.particles
        self.spec = spec
        self.device = device
        self.dim = spec.grid.dim
        self.n = p.n
        self._arrays = [np.ascontiguousarray(a, dtype=np.float64) for a in
                        (p.x, p.v, p.B, p.F, p.vol0, p.mass, p.E, p.nu)]
        flags = np.ascontiguousarray(p.flags, dtype=np.uint8)
        pin = osmpm_particles_in(p.n, *(_dp(a) for a in self._arrays),
                                 flags.ctypes.data_as(POINTER(c_uint8)))
        desc = make_desc(spec)
        self._cbs = None
        alloc_ptr = None
        if use_torch_allocator:
            alloc, self._cbs = torch_allocator(device)
            self._alloc = alloc
            alloc_ptr = ctypes.byref(alloc)
        self.stream = current_stream() if stream is None else stream
        h = c_void_p()
        _check(_lib.osmpm_create_domain(ctypes.byref(desc), ctypes.byref(pin), alloc_ptr,
                                        c_void_p(self.stream), ctypes.byref(h)),
               "osmpm_create_domain")
        self.h = h
        self.set_dirichlet(spec.dirichlet)

    # -- lifetime
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.osmpm_destroy_domain(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls
    def set_dirichlet(self, rules):
        arr = make_rules(rules)
        _check(_lib.osmpm_set_dirichlet(self.h, arr, len(rules)), "osmpm_set_dirichlet")

    def step(self, dt: float) -> dict:
        st = osmpm_stats()
        _check(_lib.osmpm_step(self.h, dt, ctypes.byref(st)), "osmpm_step")
        return st.as_dict()

    def set_plane(self, level: float = 0.0, cand_hi: float = 0.0, spacing: float = 0.0,
                  enabled: bool = True, max_sets: int = 0) -> None:
        """Rigid frictionless plane y = level (osmpm_set_plane); enabled
        False removes it."""
        pl = osmpm_plane(1 if enabled else 0, int(max_sets), float(level), float(cand_hi),
                         float(spacing))
        _check(_lib.osmpm_set_plane(self.h, ctypes.byref(pl)), "osmpm_set_plane")

    def record(self, enable: bool = True, every: int = 1) -> None:
        """Start (or with enable False stop) recording for the reverse mode;
        every >= 2 keeps a checkpoint every ``every`` steps and lets the
        adjoint re-run each segment."""
        _check(_lib.osmpm_record(self.h, max(1, int(every)) if enable else 0), "osmpm_record")

    def adjoint(self, dJ_dx, initial_state: bool = False):
        """dJ/dE for dJ_dx = dJ/dx after the recorded steps (a CUDA float64
        tensor (n, dim), id order).  Returns (dJ_dE, adjoints of the recorded
        start state as a dict of tensors when ``initial_state``, stats)."""
        import torch
        n, d = self.n, self.dim
        if dJ_dx.dtype != torch.float64 or not dJ_dx.is_cuda or tuple(dJ_dx.shape) != (n, d):
            raise ValueError("dJ_dx must be a CUDA float64 tensor of shape (n, dim)")
        g = dJ_dx.contiguous()
        torch.cuda.synchronize(g.device)
        dE = torch.empty(n, dtype=torch.float64, device=g.device)
        out = osmpm_adjoint_out()
        out.dJ_dE = dE.data_ptr()
        state = {}
        if initial_state:
            shapes = {"x": (n, d), "v": (n, d), "B": (n, d, d), "F": (n, d, d)}
            for k, shp in shapes.items():
                state[k] = torch.empty(shp, dtype=torch.float64, device=g.device)
                setattr(out, f"dJ_d{k}0", state[k].data_ptr())
        st = osmpm_stats()
        _check(_lib.osmpm_adjoint(self.h, None, c_void_p(g.data_ptr()), ctypes.byref(out),
                                  ctypes.byref(st)), "osmpm_adjoint")
        return dE, state, st.as_dict()

    def get_particles(self):
        n, d = self.n, self.dim
        x = np.empty((n, d))
        v = np.empty((n, d))
        B = np.empty((n, d, d))
        F = np.empty((n, d, d))
        _check(_lib.osmpm_get_particles(self.h, _dp(x), _dp(v), _dp(B), _dp(F)),
               "osmpm_get_particles")
        return x, v, B, F

    def set_particles(self, x, v, B, F):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, v, B, F)]
        _check(_lib.osmpm_set_particles(self.h, *(_dp(a) for a in arrs)), "osmpm_set_particles")

    def get_order(self) -> np.ndarray:
        ids = np.empty(self.n, dtype=np.uint32)
        _check(_lib.osmpm_get_order(self.h, ids.ctypes.data_as(POINTER(c_uint32))), "osmpm_get_order")
        return ids

    def get_grid(self, field: int) -> np.ndarray:
        nn = int(np.prod(self.spec.grid.res))
        comps = self.dim if field in (OSMPM_FIELD_VN, OSMPM_FIELD_U, OSMPM_FIELD_BC) else 1
        out = np.empty((nn, comps)) if comps > 1 else np.empty(nn)
        _check(_lib.osmpm_get_grid(self.h, field, _dp(out)), "osmpm_get_grid")
        return out

    def set_profiling(self, enable: bool) -> None:
        _check(_lib.osmpm_set_profiling(self.h, 1 if enable else 0), "osmpm_set_profiling")

    def counters(self) -> dict:
        c = osmpm_counters()
        _check(_lib.osmpm_get_counters(self.h, ctypes.byref(c)), "osmpm_get_counters")
        return c.as_dict()

    def probe_gradient(self, dt: float, u: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        _check(_lib.osmpm_probe_gradient(self.h, dt, _dp(u), _dp(out)), "osmpm_probe_gradient")
        return out

    def probe_hvp(self, dt: float, u: np.ndarray, d: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        out = np.empty_like(u)
        _check(_lib.osmpm_probe_hvp(self.h, dt, _dp(u), _dp(d), _dp(out)), "osmpm_probe_hvp")
        return out

    def probe_energy_change(self, dt: float, u: np.ndarray, d: np.ndarray, alpha: float) -> float:
        u = np.ascontiguousarray(u, dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        out = c_double()
        _check(_lib.osmpm_probe_energy_change(self.h, dt, _dp(u), _dp(d), alpha, ctypes.byref(out)),
               "osmpm_probe_energy_change")
        return out.value


def osmpm_create_domain(spec, stream: Optional[int] = None, use_torch_allocator: bool = True) -> Domain:
    return Domain(spec, stream, use_torch_allocator)


def osmpm_destroy_domain(dom: Domain) -> None:
    dom.close()


def osmpm_step(dom: Domain, dt: float) -> dict:
    return dom.step(dt)


def osmpm_schwarz_couple(coarse: Domain, fine: Domain, dT: float, sch) -> dict:
    """One global Schwarz step; returns the stats (``converged`` = 0 when
    k_max was reached, in which case the last iterate was committed)."""
    sd = make_schwarz_desc(sch)
    st = osmpm_stats()
    _check(_lib.osmpm_schwarz_couple(coarse.h, fine.h, dT, ctypes.byref(sd), ctypes.byref(st)),
           "osmpm_schwarz_couple", warn_ok=True)
    return st.as_dict()


def osmpm_energy_change_noalloc(grid: osmpm_noalloc_grid, parts: osmpm_noalloc_particles,
                                dt: float, alpha: float, dE_ptr: int, stream: int) -> int:
    """Raw call of the allocation-free energy change (device pointers in the
    two structs and in dE_ptr); returns the status code."""
    return _lib.osmpm_energy_change_noalloc(ctypes.byref(grid), ctypes.byref(parts), dt, alpha,
                                            c_void_p(dE_ptr), c_void_p(stream))


def osmpm_check_wait_timeout(stream: int) -> int:
    """Runs the bounded-wait diagnostic; returns the status code."""
    return _lib.osmpm_check_wait_timeout(c_void_p(stream))


def osmpm_record(dom: Domain, enable: bool = True, every: int = 1) -> None:
    dom.record(enable, every)


def osmpm_adjoint(coarse: Domain, fine: Optional[Domain], dJ_dx, initial_state: bool = False):
    """Reverse-mode gradient through the steps recorded on ``coarse`` (fine
    None) or through the pair's recorded coupled steps.  In the coupled case
    dJ_dx is a CUDA float64 tensor (n_coarse + n_fine, dim), coarse rows
    first, and every output has the same order."""
    if fine is None:
        return coarse.adjoint(dJ_dx, initial_state)
    import torch
    n, d = coarse.n + fine.n, coarse.dim
    if dJ_dx.dtype != torch.float64 or not dJ_dx.is_cuda or tuple(dJ_dx.shape) != (n, d):
        raise ValueError("dJ_dx must be a CUDA float64 tensor of shape (n_coarse + n_fine, dim)")
    g = dJ_dx.contiguous()
    torch.cuda.synchronize(g.device)
    dE = torch.empty(n, dtype=torch.float64, device=g.device)
    out = osmpm_adjoint_out()
    out.dJ_dE = dE.data_ptr()
    state = {}
    if initial_state:
        shapes = {"x": (n, d), "v": (n, d), "B": (n, d, d), "F": (n, d, d)}
        for k, shp in shapes.items():
            state[k] = torch.empty(shp, dtype=torch.float64, device=g.device)
            setattr(out, f"dJ_d{k}0", state[k].data_ptr())
    st = osmpm_stats()
    _check(_lib.osmpm_adjoint(coarse.h, fine.h, c_void_p(g.data_ptr()), ctypes.byref(out),
                              ctypes.byref(st)), "osmpm_adjoint")
    return dE, state, st.as_dict()


def _trajectory_function():
    import torch

    class Trajectory(torch.autograd.Function):
        """x_final = steps(E): n_steps backward-Euler steps of a domain built
        from ``spec`` with per-particle Young's moduli E (a float64 tensor in
        id order); backward is one osmpm_adjoint over the recorded steps."""

        @staticmethod
        def forward(ctx, E, spec, n_steps, dt):
            import dataclasses
            p = spec.particles.copy()
            p.E = E.detach().to("cpu", torch.float64).numpy().copy()
            dom = Domain(dataclasses.replace(spec, particles=p))
            dom.record(True)
            for _ in range(n_steps):
                dom.step(dt)
            x = dom.get_particles()[0]
            ctx.dom = dom
            ctx.E_device = E.device
            return torch.from_numpy(x).to(E.device)

        @staticmethod
        def backward(ctx, gx):
            dom = ctx.dom
            dE, _, _ = dom.adjoint(gx.to(f"cuda:{dom.device}", torch.float64).contiguous())
            dom.close()
            return dE.to(ctx.E_device), None, None, None

    return Trajectory


def trajectory(E, spec, n_steps: int, dt: float):
    """Differentiable final positions (n, dim) after n_steps steps of dt with
    Young's moduli E: torch.autograd.Function backed by osmpm_adjoint."""
    return _trajectory_function().apply(E, spec, n_steps, dt)


def launch_count() -> int:
    c = osmpm_counters()
    _check(_lib.osmpm_get_counters(None, ctypes.byref(c)), "osmpm_get_counters")
    return int(c.launches)


def osmpm_schwarz_couple_batch(coarse: List[Domain], fine: List[Domain], dT: float, schs,
                               n_threads: int = 8):
    """One global step of every pair (coarse[i], fine[i]) with Schwarz
    controls schs[i], pairs driven concurrently by host worker threads.
    Returns (stats list, status list)."""
    n = len(coarse)
    cs = (c_void_p * n)(*[d.h.value for d in coarse])
    fs = (c_void_p * n)(*[d.h.value for d in fine])
    sd = (osmpm_schwarz_desc * n)(*[make_schwarz_desc(s) for s in schs])
    st = (osmpm_stats * n)()
    status = (c_int32 * n)()
    _check(_lib.osmpm_schwarz_couple_batch(cs, fs, n, dT, sd, n_threads, st, status),
           "osmpm_schwarz_couple_batch", warn_ok=True)
    return [s.as_dict() for s in st], list(status)


def osmpm_schwarz_couple_multi(coarse: List[Domain], fine: List[Domain], dT: float, schs,
                               n_threads: int = 0, dof_tile: int = 0, chunk: int = 0,
                               slot_tiles: int = 0):
    """One global step of every pair (mixed precision) with the batched PCG
    service: host threads drive the pairs, every Newton system is solved in a
    batched PCG together with the systems of the other pairs.  Returns
    (stats list, status list, service counters)."""
    n = len(coarse)
    cs = (c_void_p * n)(*[d.h.value for d in coarse])
    fs = (c_void_p * n)(*[d.h.value for d in fine])
    sd = (osmpm_schwarz_desc * n)(*[make_schwarz_desc(s) for s in schs])
    st = (osmpm_stats * n)()
    status = (c_int32 * n)()
    md = osmpm_multi_desc(int(n_threads), int(dof_tile), int(chunk), int(slot_tiles))
    ms = osmpm_multi_stats()
    _check(_lib.osmpm_schwarz_couple_multi(cs, fs, n, dT, sd, ctypes.byref(md), st, status,
                                           ctypes.byref(ms)),
           "osmpm_schwarz_couple_multi", warn_ok=True)
    return [s.as_dict() for s in st], list(status), ms.as_dict()


def osmpm_autotune_multi(coarse: List[Domain], fine: List[Domain], dT: float, schs, candidates):
    """Launch shape of osmpm_schwarz_couple_multi chosen by timing one step
    per candidate, each a (n_threads, dof_tile, chunk[, slot_tiles]) tuple
    (the pairs advance by len(candidates) + 1 global steps).  Returns (best
    candidate, list of wall microseconds per PCG iteration)."""
    n = len(coarse)
    cs = (c_void_p * n)(*[d.h.value for d in coarse])
    fs = (c_void_p * n)(*[d.h.value for d in fine])
    sd = (osmpm_schwarz_desc * n)(*[make_schwarz_desc(s) for s in schs])
    cand = (osmpm_multi_desc * len(candidates))(
        *[osmpm_multi_desc(*[int(v) for v in (tuple(c) + (0,))[:4]]) for c in candidates])
    best = c_int32(0)
    score = np.zeros(len(candidates), dtype=np.float64)
    _check(_lib.osmpm_autotune_multi(cs, fs, n, dT, sd, cand, len(candidates), ctypes.byref(best),
                                     score.ctypes.data_as(_DP)),
           "osmpm_autotune_multi", warn_ok=True)
    return tuple(candidates[int(best.value)]), [float(v) for v in score]


def create_stream() -> int:
    """A new non-blocking CUDA stream made by the library (a distinct stream
    per pair of osmpm_schwarz_couple_batch; torch.cuda.Stream() hands out
    streams from a fixed pool).  Release with destroy_stream."""
    h = c_void_p()
    _check(_lib.osmpm_create_stream(ctypes.byref(h)), "osmpm_create_stream")
    return int(h.value)


def destroy_stream(stream: int) -> None:
    _check(_lib.osmpm_destroy_stream(c_void_p(stream)), "osmpm_destroy_stream")


def osmpm_autotune_batch(coarse: List[Domain], fine: List[Domain], dT: float, schs, candidates):
    """Host concurrency for osmpm_schwarz_couple_batch on these pairs, chosen
    by timing one batched step per candidate (the pairs advance by
    len(candidates) + 1 global steps).  Returns (best, {candidate: wall
    microseconds per PCG iteration})."""
    n = len(coarse)
    cs = (c_void_p * n)(*[d.h.value for d in coarse])
    fs = (c_void_p * n)(*[d.h.value for d in fine])
    sd = (osmpm_schwarz_desc * n)(*[make_schwarz_desc(s) for s in schs])
    cand = (c_int32 * len(candidates))(*candidates)
    best = c_int32(0)
    score = np.zeros(len(candidates), dtype=np.float64)
    _check(_lib.osmpm_autotune_batch(cs, fs, n, dT, sd, cand, len(candidates), ctypes.byref(best),
                                     score.ctypes.data_as(_DP)),
           "osmpm_autotune_batch", warn_ok=True)
    return int(best.value), {int(c): float(v) for c, v in zip(candidates, score)}


def osmpm_get_particles(dom: Domain):
    return dom.get_particles()


def osmpm_set_particles(dom: Domain, x, v, B, F):
    dom.set_particles(x, v, B, F)


def osmpm_get_order(dom: Domain):
    return dom.get_order()


def osmpm_get_grid(dom: Domain, field: int):
    return dom.get_grid(field)
