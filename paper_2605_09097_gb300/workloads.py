"""Seeded synthetic inputs for the OS-MPM hot path.

This module builds particle sets, background grids, Dirichlet rules and
coupling parameters for the paper's numerical examples (Sec. 4) and for the
small unit cases the tests use.  It is the one module that both the CUDA path
and the FP64 CPU oracle read, so it holds none of the method's arithmetic:
no shape functions, no transfers, no constitutive law, no solver.  Everything
here is geometry (which lattice points lie in which region), bookkeeping
(particle volume and mass from the cell size and density) and seeded random
perturbations.

Particle sampling follows one fixed rule (used everywhere): a regular lattice
of ``ppc_1d**d`` points per grid cell at offsets ``(q + 1/2) / ppc_1d`` of the
cell, kept when the point lies inside the material region (half-open boxes,
``r < R`` for disks).  Creation order is cells with x fastest (then y, then z)
and, inside a cell, sub-points with x fastest; that order is the stable
particle id.  ``V0 = dx**d / ppc``, ``m = rho * V0``.
"""
from __future__ import annotations

import dataclasses
import itertools
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

BIG = 1.0e30  # stands for an unbounded side of a Dirichlet box

FLAG_BOUNDARY = 1  # bit 0: particle belongs to the boundary layer P_alpha^partial (Sec. 3.2.1)


@dataclass
class Grid:
    dim: int
    origin: Tuple[float, ...]
    dx: float
    res: Tuple[int, ...]

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.res))


@dataclass
class Dirichlet:
    """Prescribed grid-node velocity on the nodes whose position lies in the
    closed box [lo, hi].  ``kind`` 0: uniform velocity ``vel`` on the
    components in ``comp_mask`` (bit c = component c).  ``kind`` 1: rigid
    rotation about the axis through ``center`` along ``axis`` (3D; in 2D the
    axis is z) by ``omega`` radians per unit time, all components."""

    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    comp_mask: int = 0b111
    vel: Tuple[float, ...] = (0.0, 0.0, 0.0)
    kind: int = 0
    center: Tuple[float, ...] = (0.0, 0.0, 0.0)
    axis: Tuple[float, ...] = (0.0, 0.0, 1.0)
    omega: float = 0.0


@dataclass
class Particles:
    x: np.ndarray      # (N, d) float64
    v: np.ndarray      # (N, d)
    B: np.ndarray      # (N, d, d) APIC affine matrix
    F: np.ndarray      # (N, d, d) deformation gradient
    vol0: np.ndarray   # (N,)
    mass: np.ndarray   # (N,)
    E: np.ndarray      # (N,) Young's modulus
    nu: np.ndarray     # (N,) Poisson's ratio
    flags: np.ndarray  # (N,) uint8

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def copy(self) -> "Particles":
        return Particles(*(np.array(getattr(self, f.name), copy=True)
                           for f in dataclasses.fields(self)))


@dataclass
class DomainSpec:
    name: str
    grid: Grid
    particles: Particles
    gravity: Tuple[float, ...]
    dirichlet: List[Dirichlet] = field(default_factory=list)
    newton_tol: float = 1e-8      # on max |delta x_hat| / dt  (m/s)
    newton_max: int = 100
    cg_rtol: float = 1e-6
    cg_max: int = 20000
    ls_max: int = 40
    # nodes with m_i <= mass_eps carry no DOF; None -> 1e-10 x mean particle mass
    mass_eps: Optional[float] = None
    precision: int = 0            # 0: FP64; 1: mixed (FP32 particle state and HVP)
    cg_eta_max: float = 0.0       # inexact-Newton forcing cap (0: the library default 1e-3)
    pcg_mode: int = 0             # 0 automatic, 1 persistent PCG, 2 streaming PCG
    launch_mode: int = 0          # 0 CUDA graph per Newton iteration, 1 plain stream launches
    hvp_mode: int = 0             # mixed streaming PCG product: 0 automatic, 1 lane groups, 2 tiles

    def __post_init__(self):
        if self.mass_eps is None:
            self.mass_eps = 1e-10 * float(np.mean(self.particles.mass))


@dataclass
class SchwarzSpec:
    M: int                # sub-cycling ratio dT / dt (Sec. 3.1)
    k_max: int = 50       # Schwarz iteration cap (Alg. 1)
    eps_conv: float = 1e-5   # Sec. 4: tolerance of the interface residuals
    tau_B: float = 0.0    # boundary-node mass threshold on the coarse grid
    tau_S: float = 0.0    # same on the fine grid
    eps_tol: float = 0.0  # projection regulariser (Eq. spatial_projection)
    pi_source: int = 0    # fine state projected for k >= 1: 0 step average, 1 last sub-step's P2G


# ----------------------------------------------------------------------------
# lattice sampling
# ----------------------------------------------------------------------------

def sample_lattice(origin: Sequence[float], dx: float,
                   cell_lo: Sequence[int], cell_hi: Sequence[int],
                   ppc_1d: int,
                   inside: Callable[[np.ndarray], np.ndarray]) -> np.ndarray:
    """Lattice points of cells ``cell_lo <= c < cell_hi`` (per axis) of the
    grid with ``origin`` and ``dx``; returns the kept points (K, d) in creation
    order."""
    d = len(origin)
    origin = np.asarray(origin, dtype=np.float64)
    # cells, x fastest
    axes_c = [np.arange(cell_lo[a], cell_hi[a]) for a in range(d)]
    cells = np.stack(np.meshgrid(*axes_c[::-1], indexing="ij")[::-1], axis=-1).reshape(-1, d)
    q = np.arange(ppc_1d)
    subs = np.stack(np.meshgrid(*([q] * d), indexing="ij")[::-1], axis=-1).reshape(-1, d)
    off = (subs + 0.5) / ppc_1d
    pts = (cells[:, None, :] + off[None, :, :]).reshape(-1, d)
    x = origin[None, :] + pts * dx
    keep = inside(x)
    return np.ascontiguousarray(x[keep])


def make_particles(x: np.ndarray, dx: float, ppc_1d: int, rho: float,
                   E: np.ndarray, nu: np.ndarray,
                   flags: Optional[np.ndarray] = None,
                   F0: Optional[np.ndarray] = None) -> Particles:
    n, d = x.shape
    vol = dx ** d / ppc_1d ** d
    F = np.broadcast_to(np.eye(d), (n, d, d)).copy() if F0 is None else np.array(F0, dtype=np.float64)
    return Particles(
        x=np.array(x, dtype=np.float64),
        v=np.zeros((n, d)),
        B=np.zeros((n, d, d)),
        F=F,
        vol0=np.full(n, vol),
        mass=np.full(n, rho * vol),
        E=np.broadcast_to(np.asarray(E, dtype=np.float64), (n,)).copy(),
        nu=np.broadcast_to(np.asarray(nu, dtype=np.float64), (n,)).copy(),
        flags=np.zeros(n, np.uint8) if flags is None else flags.astype(np.uint8),
    )


def _box(lo, hi):
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lambda x: np.all((x >= lo) & (x < hi), axis=1)


def _r2(x, c):
    c = np.asarray(c, dtype=np.float64)
    return np.sum((x - c[None, :]) ** 2, axis=1)


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------

def cantilever(dx: float = 0.0125, ppc_1d: int = 2, L: float = 1.0, H: float = 0.1,
               E: float = 1e6, nu: float = 0.3, rho: float = 1000.0,
               g: float = -9.81, origin=(-0.1, -1.0), res=(112, 96),
               newton_tol: float = 1e-8) -> DomainSpec:
    """2D cantilever beam [0,L]x[0,H] clamped at x=0 under gravity (Sec. 4.1
    geometry; single domain).  The clamp fixes every grid node with x_i <= 0."""
    nc = (int(round(L / dx)), int(round(H / dx)))
    x = sample_lattice((0.0, 0.0), dx, (0, 0), nc, ppc_1d, _box((0.0, 0.0), (L, H)))
    p = make_particles(x, dx, ppc_1d, rho, E, nu)
    grid = Grid(2, tuple(origin), dx, tuple(res))
    clamp = Dirichlet(lo=(-BIG, -BIG), hi=(0.5 * dx, BIG), comp_mask=0b11)
    return DomainSpec("cantilever", grid, p, (0.0, g), [clamp], newton_tol=newton_tol)


def eb_gravity(gamma: float, L=1.0, H=0.1, E=1e6, nu=0.3, rho=1000.0) -> float:
    """Gravity that gives gravito-bending number ``gamma`` for a plane-strain
    beam of height H and unit width: Gamma = rho g H L^3 / D,
    D = E H^3 / (12 (1 - nu^2))  (Sec. 4.1)."""
    D = E * H ** 3 / (12.0 * (1.0 - nu ** 2))
    return gamma * D / (rho * H * L ** 3)


def inclusion(dx_S: float = 0.005, M: int = 2, dx_B: float = 0.05,
              r_inc: float = 0.05, E_inc: float = 1e8, E: float = 1e6, nu: float = 0.3,
              rho: float = 1000.0, dT: float = 0.01, top_disp: float = 1e-3,
              r_hole: float = 0.1, r_fine: float = 0.15, ppc_1d: int = 2,
              newton_tol: float = 1e-8, cg_rtol: float = 1e-6, eigenstrain: float = 0.0,
              free_edges: bool = False):
    """2D elastic inclusion for OS-MPM (Sec. 4.3 geometry with a displaced top
    edge).  Coarse: matrix [0.1,0.9]^2 minus the disk r < r_hole on the grid
    [0,1]^2 at dx_B.  Fine: disk r < r_fine on the grid [0.3,0.7]^2 at dx_S
    (wider when r_fine + 4 dx_S exceeds 0.2),
    with the stiff inclusion r < r_inc.  ``eigenstrain`` delta > 0 starts the
    inclusion particles at F0 = (1 - delta) I (the loading of Sec. 4.3).
    The matrix's bottom edge is clamped and its top edge moves by
    ``top_disp`` in y over dT; ``free_edges`` drops both rules (the traction-
    free matrix of the eigenstrain problem).  Returns (coarse, fine, schwarz, dT)."""
    c = (0.5, 0.5)
    # coarse domain
    nB = int(round(1.0 / dx_B)) + 1
    gB = Grid(2, (0.0, 0.0), dx_B, (nB, nB))
    lo_c = int(round(0.1 / dx_B))
    hi_c = int(round(0.9 / dx_B))
    xB = sample_lattice(gB.origin, dx_B, (lo_c, lo_c), (hi_c, hi_c), ppc_1d,
                        lambda x: _box((0.1, 0.1), (0.9, 0.9))(x) & (_r2(x, c) >= r_hole ** 2))
    sB = dx_B / ppc_1d
    flB = np.where(_r2(xB, c) < (r_hole + sB) ** 2, FLAG_BOUNDARY, 0).astype(np.uint8)
    pB = make_particles(xB, dx_B, ppc_1d, rho, E, nu, flB)
    v_top = -top_disp / dT
    dirB = [] if free_edges else [
        Dirichlet(lo=(-BIG, -BIG), hi=(BIG, 0.1 + 0.5 * dx_B), comp_mask=0b11),
        Dirichlet(lo=(-BIG, 0.9 - 0.5 * dx_B), hi=(BIG, BIG), comp_mask=0b10, vel=(0.0, v_top, 0.0)),
    ]
    coarse = DomainSpec("inclusion_coarse", gB, pB, (0.0, 0.0), dirB,
                        newton_tol=newton_tol, cg_rtol=cg_rtol)
    # fine domain
    # fine grid: the square [0.3, 0.7]^2, widened when the disk needs it
    half = max(0.2, float(np.ceil((r_fine + 4 * dx_S) / dx_S - 1e-9)) * dx_S)
    nS = int(round(2 * half / dx_S)) + 1
    gS = Grid(2, (0.5 - half, 0.5 - half), dx_S, (nS, nS))
    ncS = nS - 1
    xS = sample_lattice(gS.origin, dx_S, (0, 0), (ncS, ncS), ppc_1d,
                        lambda x: _r2(x, c) < r_fine ** 2)
    sS = dx_S / ppc_1d
    flS = np.where(_r2(xS, c) >= (r_fine - sS) ** 2, FLAG_BOUNDARY, 0).astype(np.uint8)
    inc = _r2(xS, c) < r_inc ** 2
    Es = np.where(inc, E_inc, E)
    F0 = np.broadcast_to(np.eye(2), (xS.shape[0], 2, 2)).copy()
    F0[inc] *= (1.0 - eigenstrain)
    pS = make_particles(xS, dx_S, ppc_1d, rho, Es, nu, flS, F0=F0)
    fine = DomainSpec("inclusion_fine", gS, pS, (0.0, 0.0), [],
                      newton_tol=newton_tol, cg_rtol=cg_rtol)
    sch = SchwarzSpec(M=M, k_max=50, eps_conv=1e-5,
                      tau_B=rho * dx_B ** 2 / ppc_1d ** 2,
                      tau_S=rho * dx_S ** 2 / ppc_1d ** 2,
                      eps_tol=1e-12 * rho * dx_S ** 2)
    return coarse, fine, sch, dT


def inclusion_single(dx: float = 0.005, r_inc: float = 0.05, E_inc: float = 1e6,
                     E: float = 1e6, nu: float = 0.3, rho: float = 1000.0,
                     eigenstrain: float = 0.01, ppc_1d: int = 2, newton_tol: float = 1e-8,
                     cg_rtol: float = 1e-6) -> DomainSpec:
    """The single-domain reference of Sec. 4.3: the traction-free matrix
    [0.1,0.9]^2 with the inclusion r < r_inc (F0 = (1 - eigenstrain) I,
    modulus E_inc) on one grid [0,1]^2 at dx."""
    c = (0.5, 0.5)
    n = int(round(1.0 / dx)) + 1
    g = Grid(2, (0.0, 0.0), dx, (n, n))
    lo, hi = int(round(0.1 / dx)), int(round(0.9 / dx))
    x = sample_lattice(g.origin, dx, (lo, lo), (hi, hi), ppc_1d, _box((0.1, 0.1), (0.9, 0.9)))
    inc = _r2(x, c) < r_inc ** 2
    F0 = np.broadcast_to(np.eye(2), (x.shape[0], 2, 2)).copy()
    F0[inc] *= (1.0 - eigenstrain)
    p = make_particles(x, dx, ppc_1d, rho, np.where(inc, E_inc, E), nu, F0=F0)
    return DomainSpec("inclusion_single", g, p, (0.0, 0.0), [], newton_tol=newton_tol,
                      cg_rtol=cg_rtol)


def hertz(dx_c: float = 1.0 / 64, ratio: int = 4, M: int = 4, E_block: float = 1e6,
          E_cyl: float = 1e7, nu: float = 0.3, rho: float = 1000.0, R: float = 0.5,
          dT: float = 2e-4, indent: float = 0.02, n_steps: int = 100, ppc_1d: int = 2,
          box_lo=(1.75, 1.875), box_hi=(2.25, 2.125), precision: int = 1,
          newton_tol: float = 1e-8, cg_rtol: float = 1e-6):
    """2D Hertzian contact for OS-MPM (Sec. 4.2 setting with an elastic
    block instead of the rigid plane): block [0,4]x[0,2] on a coarse grid
    covering [0,4]x[0,3] plus a 3-cell margin, half-disk cylinder
    r < R, y < 2 + R centred at (2, 2 + R) (flat face up, lowest point
    touching the block top at (2, 2)), both on one grid per domain.  The
    cylinder's flat face is pushed down by ``indent`` over ``n_steps`` global
    steps of dT; the block bottom is fixed.  Fine subdomain: the box
    [box_lo, box_hi] at dx_c / ratio; coarse: all material minus the box
    shrunk by 2 dx_c.  Returns (coarse, fine, schwarz, dT)."""
    c = np.array([2.0, 2.0 + R])
    dx_f = dx_c / ratio
    blo, bhi = np.asarray(box_lo), np.asarray(box_hi)

    def body(x):
        in_block = np.all((x >= 0.0) & (x < np.array([4.0, 2.0])), axis=1)
        in_cyl = (_r2(x, c) < R * R) & (x[:, 1] < c[1])
        return in_block, in_cyl

    def in_box(x, lo, hi):
        return np.all((x >= lo) & (x < hi), axis=1)

    hole_lo, hole_hi = blo + 2 * dx_c, bhi - 2 * dx_c
    # coarse domain on [0,4] x [0,3] with a 3-cell margin
    nBx, nBy = int(round(4.0 / dx_c)), int(round(3.0 / dx_c))
    mB = 3
    gB = Grid(2, (-mB * dx_c, -mB * dx_c), dx_c, (nBx + 2 * mB + 1, nBy + 2 * mB + 1))

    def coarse_in(x):
        a, b = body(x)
        return (a | b) & ~in_box(x, hole_lo, hole_hi)
    xB = sample_lattice((0.0, 0.0), dx_c, (0, 0), (nBx, nBy), ppc_1d, coarse_in)
    sB = dx_c / ppc_1d
    flB = np.where(in_box(xB, hole_lo - sB, hole_hi + sB), FLAG_BOUNDARY, 0).astype(np.uint8)
    EB = np.where(body(xB)[1], E_cyl, E_block)
    pB = make_particles(xB, dx_c, ppc_1d, rho, EB, nu, flB)
    v_push = -indent / (n_steps * dT)
    dirB = [
        Dirichlet(lo=(-BIG, -BIG), hi=(BIG, 0.5 * dx_c), comp_mask=0b11),
        Dirichlet(lo=(-BIG, c[1] - 0.5 * dx_c), hi=(BIG, BIG), comp_mask=0b11,
                  vel=(0.0, v_push, 0.0)),
    ]
    coarse = DomainSpec("hertz_coarse", gB, pB, (0.0, 0.0), dirB, newton_tol=newton_tol,
                        cg_rtol=cg_rtol, precision=precision)
    # fine domain: the box with a 3-cell margin
    margin = 3
    o = tuple(blo - margin * dx_f)
    nfx = int(round((bhi[0] - blo[0]) / dx_f)) + 2 * margin
    nfy = int(round((bhi[1] - blo[1]) / dx_f)) + 2 * margin
    gS = Grid(2, o, dx_f, (nfx + 1, nfy + 1))

    def fine_in(x):
        a, b = body(x)
        return (a | b) & in_box(x, blo, bhi)
    xS = sample_lattice(o, dx_f, (0, 0), (nfx, nfy), ppc_1d, fine_in)
    sS = dx_f / ppc_1d
    flS = np.where(~in_box(xS, blo + sS, bhi - sS), FLAG_BOUNDARY, 0).astype(np.uint8)
    ES = np.where(body(xS)[1], E_cyl, E_block)
    pS = make_particles(xS, dx_f, ppc_1d, rho, ES, nu, flS)
    fine = DomainSpec("hertz_fine", gS, pS, (0.0, 0.0), [], newton_tol=newton_tol,
                      cg_rtol=cg_rtol, precision=precision)
    sch = SchwarzSpec(M=M, k_max=50, eps_conv=1e-5,
                      tau_B=rho * dx_c ** 2 / ppc_1d ** 2, tau_S=rho * dx_f ** 2 / ppc_1d ** 2,
                      eps_tol=1e-12 * rho * dx_f ** 2)
    return coarse, fine, sch, dT


def hertz_rigid(dx_c: float = 1.0 / 64, ratio: int = 4, M: int = 4, E: float = 2e5,
                nu: float = 0.3, rho: float = 1000.0, R: float = 0.5, dT: float = 0.02,
                indent: float = 0.01, n_steps: int = 10, ppc_1d: int = 2,
                box_half=(0.25, 0.125), precision: int = 0, newton_tol: float = 1e-8,
                cg_rtol: float = 1e-6):
    """The Hertz benchmark of Sec. 4.2: a half-disk cylinder r < R, y < R
    centred at (0, R) (flat face up, lowest point touching the plane y = 0)
    pressed onto a rigid frictionless plane.  The plane is the grid nodes
    with y <= 0, whose y velocity is held at zero (x free); the flat face's
    nodes move down by ``indent`` over ``n_steps`` global steps of dT.  Fine
    subdomain: the box [-bx, bx] x [0, by] around the contact at dx_c /
    ratio; coarse: the cylinder minus that box shrunk by 2 dx_c.  Returns
    (coarse, fine, schwarz, dT)."""
    c = np.array([0.0, R])
    dx_f = dx_c / ratio
    blo = np.array([-box_half[0], 0.0])
    bhi = np.array([box_half[0], box_half[1]])

    def cyl(x):
        return (_r2(x, c) < R * R) & (x[:, 1] < c[1])

    def in_box(x, lo, hi):
        return np.all((x >= lo) & (x < hi), axis=1)

    hole_lo, hole_hi = blo + np.array([2 * dx_c, -BIG]), bhi - 2 * dx_c
    m = 3
    nx = int(round(2 * (R + 0.05) / dx_c))
    ny = int(round((R + 0.05) / dx_c))
    gB = Grid(2, (-(R + 0.05) - m * dx_c, -m * dx_c), dx_c, (nx + 2 * m + 1, ny + 2 * m + 1))
    xB = sample_lattice(gB.origin, dx_c, (m, m), (m + nx, m + ny), ppc_1d,
                        lambda x: cyl(x) & ~in_box(x, hole_lo, hole_hi))
    sB = dx_c / ppc_1d
    flB = np.where(in_box(xB, hole_lo - sB, hole_hi + sB), FLAG_BOUNDARY, 0).astype(np.uint8)
    pB = make_particles(xB, dx_c, ppc_1d, rho, E, nu, flB)
    v_push = -indent / (n_steps * dT)
    plane = lambda dx: Dirichlet(lo=(-BIG, -BIG), hi=(BIG, 0.5 * dx), comp_mask=0b10)
    top = Dirichlet(lo=(-BIG, R - 0.5 * dx_c), hi=(BIG, BIG), comp_mask=0b11, vel=(0.0, v_push, 0.0))
    coarse = DomainSpec("hertz_rigid_coarse", gB, pB, (0.0, 0.0), [plane(dx_c), top],
                        newton_tol=newton_tol, cg_rtol=cg_rtol, precision=precision)
    mf = 3
    nfx = int(round((bhi[0] - blo[0]) / dx_f))
    nfy = int(round((bhi[1] - blo[1]) / dx_f))
    o = (blo[0] - mf * dx_f, blo[1] - mf * dx_f)
    gS = Grid(2, o, dx_f, (nfx + 2 * mf + 1, nfy + 2 * mf + 1))
    xS = sample_lattice(o, dx_f, (mf, mf), (mf + nfx, mf + nfy), ppc_1d,
                        lambda x: cyl(x) & in_box(x, blo, bhi))
    sS = dx_f / ppc_1d
    inner = in_box(xS, blo + np.array([sS, -BIG]), bhi - sS)
    flS = np.where(~inner, FLAG_BOUNDARY, 0).astype(np.uint8)
    pS = make_particles(xS, dx_f, ppc_1d, rho, E, nu, flS)
    fine = DomainSpec("hertz_rigid_fine", gS, pS, (0.0, 0.0), [plane(dx_f)],
                      newton_tol=newton_tol, cg_rtol=cg_rtol, precision=precision)
    sch = SchwarzSpec(M=M, k_max=50, eps_conv=1e-5,
                      tau_B=rho * dx_c ** 2 / ppc_1d ** 2, tau_S=rho * dx_f ** 2 / ppc_1d ** 2,
                      eps_tol=1e-12 * rho * dx_f ** 2)
    return coarse, fine, sch, dT


def hertz_rigid_single(dx: float = 1.0 / 64, E: float = 2e5, nu: float = 0.3,
                       rho: float = 1000.0, R: float = 0.5, dt: float = 0.02,
                       indent: float = 0.01, n_steps: int = 10, ppc_1d: int = 2,
                       newton_tol: float = 1e-8):
    """The cylinder of the Sec. 4.2 benchmark on one grid at dx: the
    half-disk r < R, y < R centred at (0, R), lowest point on the plane
    y = 0; its flat face's nodes move down by ``indent`` over ``n_steps``
    steps of dt (that rule is the spec's only Dirichlet entry, so a caller
    can stop the push by zeroing its velocity).  The plane itself is not a Dirichlet rule here:
    the grid nodes with y <= dx/2 are the candidates of a unilateral
    contact (``plane_nodes``).  Returns (spec, plane_nodes)."""
    c = np.array([0.0, R])

    def cyl(x):
        return (_r2(x, c) < R * R) & (x[:, 1] < c[1])

    m = 3
    nh = int(np.ceil((R + 0.05) / dx))   # a node at x = 0: grid and lattice symmetric about the contact
    ny = int(round((R + 0.05) / dx))
    g = Grid(2, (-(nh + m) * dx, -m * dx), dx, (2 * (nh + m) + 1, ny + 2 * m + 1))
    x = sample_lattice(g.origin, dx, (m, m), (m + 2 * nh, m + ny), ppc_1d, cyl)
    p = make_particles(x, dx, ppc_1d, rho, E, nu)
    v_push = -indent / (n_steps * dt)
    top = Dirichlet(lo=(-BIG, R - 0.5 * dx), hi=(BIG, BIG), comp_mask=0b11, vel=(0.0, v_push, 0.0))
    spec = DomainSpec("hertz_rigid_single", g, p, (0.0, 0.0), [top], newton_tol=newton_tol)
    iy = np.arange(g.res[0] * g.res[1]) // g.res[0]
    plane_nodes = g.origin[1] + iy * dx <= 0.5 * dx
    return spec, plane_nodes


def fold3d(dx_c: float = 0.02, dx_f: float = 0.005, band=(0.4, 0.6), M: int = 4,
           size=(1.0, 0.5, 0.02), E: float = 1e6, nu: float = 0.3, rho: float = 1000.0,
           dT: float = 0.01, fold_steps: int = 400, ppc_1d: int = 2, precision: int = 1,
           newton_tol: float = 1e-8, cg_rtol: float = 1e-6):
    """3D folding plate for OS-MPM: plate [0,Lx]x[0,Ly]x[0,Lz], grid nodes
    with x <= 0 clamped, nodes with x >= Lx - dx_c rotated rigidly about the
    fold axis (x = (band_lo + band_hi)/2, z = Lz/2, parallel to y) by
    90 degrees over ``fold_steps`` global steps.  Fine subdomain: the band
    band_lo <= x < band_hi at dx_f; coarse: the plate minus the band shrunk
    by 2 dx_c.  The edge rule is a fixed box, so it holds the edge while the
    edge still lies in it (the first steps of the fold).  Returns
    (coarse, fine, schwarz, dT)."""
    Lx, Ly, Lz = size
    b0, b1 = band
    axis_x = 0.5 * (b0 + b1)
    hole = (b0 + 2 * dx_c, b1 - 2 * dx_c)
    m = 3

    def plate(x):
        return np.all((x >= 0.0) & (x < np.array([Lx, Ly, Lz])), axis=1)

    ncB = (int(round(Lx / dx_c)), int(round(Ly / dx_c)), max(1, int(round(Lz / dx_c))))
    gB = Grid(3, (-m * dx_c,) * 3, dx_c, tuple(n + 2 * m + 1 for n in ncB))
    xB = sample_lattice((0.0, 0.0, 0.0), dx_c, (0, 0, 0), ncB, ppc_1d,
                        lambda x: plate(x) & ~((x[:, 0] >= hole[0]) & (x[:, 0] < hole[1])))
    sB = dx_c / ppc_1d
    flB = ((xB[:, 0] >= hole[0] - sB) & (xB[:, 0] < hole[1] + sB)).astype(np.uint8)
    pB = make_particles(xB, dx_c, ppc_1d, rho, E, nu, flB)
    omega = (0.5 * np.pi) / (fold_steps * dT)
    dirB = [
        Dirichlet(lo=(-BIG, -BIG, -BIG), hi=(0.5 * dx_c, BIG, BIG), comp_mask=0b111),
        Dirichlet(lo=(Lx - dx_c - 0.5 * dx_c, -BIG, -BIG), hi=(BIG, BIG, BIG), kind=1,
                  center=(axis_x, 0.0, 0.5 * Lz), axis=(0.0, 1.0, 0.0), omega=-omega),
    ]
    coarse = DomainSpec("fold3d_coarse", gB, pB, (0.0, 0.0, 0.0), dirB,
                        newton_tol=newton_tol, cg_rtol=cg_rtol, precision=precision)
    ncS = (int(round((b1 - b0) / dx_f)), int(round(Ly / dx_f)), int(round(Lz / dx_f)))
    oS = (b0 - m * dx_f, -m * dx_f, -m * dx_f)
    gS = Grid(3, oS, dx_f, tuple(n + 2 * m + 1 for n in ncS))
    xS = sample_lattice((b0, 0.0, 0.0), dx_f, (0, 0, 0), ncS, ppc_1d, plate)
    sS = dx_f / ppc_1d
    flS = ((xS[:, 0] < b0 + sS) | (xS[:, 0] >= b1 - sS)).astype(np.uint8)
    pS = make_particles(xS, dx_f, ppc_1d, rho, E, nu, flS)
    fine = DomainSpec("fold3d_fine", gS, pS, (0.0, 0.0, 0.0), [],
                      newton_tol=newton_tol, cg_rtol=cg_rtol, precision=precision)
    sch = SchwarzSpec(M=M, k_max=50, eps_conv=1e-5,
                      tau_B=rho * dx_c ** 3 / ppc_1d ** 3, tau_S=rho * dx_f ** 3 / ppc_1d ** 3,
                      eps_tol=1e-12 * rho * dx_f ** 3)
    return coarse, fine, sch, dT


def fold3d_small(precision: int = 1, **kw):
    """A reduced 3D folding plate small enough for the FP64 oracle: plate
    0.48 x 0.12 x 0.04, coarse dx 0.04, fine band [0.12, 0.36) at dx 0.02,
    M = 2, the edge rotated 90 degrees over 20 global steps (the same rules
    and kernels as ``fold3d``: the kind-1 rotation rule, 3D, mixed precision
    by default).  240 coarse and 1,152 fine particles."""
    args = dict(dx_c=0.04, dx_f=0.02, band=(0.12, 0.36), size=(0.48, 0.12, 0.04), M=2,
                fold_steps=20, precision=precision)
    args.update(kw)
    return fold3d(**args)


def overlap3d(dx_c: float = 0.1, ratio: int = 2, M: int = 2, E: float = 1e5, nu: float = 0.3,
              rho: float = 1000.0, dT: float = 0.02, ppc_1d: int = 2, precision: int = 0):
    """A small clamped 3D bar [0,0.8]x[0,0.2]x[0,0.2] under gravity split in
    x: coarse (dx_c) covers x < 0.45, fine (dx_c/ratio) covers x >= 0.3;
    boundary layers at the artificial faces x = 0.45 (coarse) and x = 0.3
    (fine).  Small enough for the 3D oracle.  Returns (coarse, fine,
    schwarz, dT)."""
    dx_f = dx_c / ratio
    Lx, Ly, Lz = 0.8, 0.2, 0.2
    xc, xf = 0.45, 0.3
    m = 3

    def bar(x):
        return np.all((x >= 0.0) & (x < np.array([Lx, Ly, Lz])), axis=1)

    ncB = (int(round(Lx / dx_c)), int(round(Ly / dx_c)), int(round(Lz / dx_c)))
    gB = Grid(3, (-m * dx_c,) * 3, dx_c, tuple(n + 2 * m + 1 for n in ncB))
    xB = sample_lattice((0.0, 0.0, 0.0), dx_c, (0, 0, 0), ncB, ppc_1d,
                        lambda x: bar(x) & (x[:, 0] < xc))
    flB = (xB[:, 0] >= xc - dx_c / ppc_1d).astype(np.uint8)
    pB = make_particles(xB, dx_c, ppc_1d, rho, E, nu, flB)
    g = (0.0, 0.0, -9.81)
    coarse = DomainSpec("overlap3d_coarse", gB, pB, g,
                        [Dirichlet(lo=(-BIG,) * 3, hi=(0.5 * dx_c, BIG, BIG), comp_mask=0b111)],
                        precision=precision)
    ncS = (int(round((Lx - xf) / dx_f)), int(round(Ly / dx_f)), int(round(Lz / dx_f)))
    gS = Grid(3, (xf - m * dx_f, -m * dx_f, -m * dx_f), dx_f, tuple(n + 2 * m + 1 for n in ncS))
    xS = sample_lattice((xf, 0.0, 0.0), dx_f, (0, 0, 0), ncS, ppc_1d, bar)
    flS = (xS[:, 0] < xf + dx_f / ppc_1d).astype(np.uint8)
    pS = make_particles(xS, dx_f, ppc_1d, rho, E, nu, flS)
    fine = DomainSpec("overlap3d_fine", gS, pS, g, [], precision=precision)
    sch = SchwarzSpec(M=M, k_max=50, eps_conv=1e-5,
                      tau_B=rho * dx_c ** 3 / ppc_1d ** 3, tau_S=rho * dx_f ** 3 / ppc_1d ** 3,
                      eps_tol=1e-12 * rho * dx_f ** 3)
    return coarse, fine, sch, dT


def block(dim: int = 2, n_cells=(6, 5), dx: float = 0.1, ppc_1d: int = 2,
          E: float = 1e5, nu: float = 0.3, rho: float = 1000.0, margin: int = 3,
          gravity=None) -> DomainSpec:
    """A box of material of n_cells cells starting at the origin, with a grid
    that leaves ``margin`` empty cells on every side.  No Dirichlet rules."""
    nc = tuple(n_cells[:dim])
    x = sample_lattice((0.0,) * dim, dx, (0,) * dim, nc, ppc_1d,
                       _box((0.0,) * dim, tuple(n * dx for n in nc)))
    p = make_particles(x, dx, ppc_1d, rho, E, nu)
    origin = tuple(-margin * dx for _ in range(dim))
    res = tuple(n + 2 * margin + 1 for n in nc)
    g = tuple(gravity) if gravity is not None else (0.0,) * dim
    return DomainSpec(f"block{dim}d", Grid(dim, origin, dx, res), p, g, [])


def perturb(spec: DomainSpec, seed: int, v_scale=0.1, B_scale=0.0025, F_scale=0.02) -> DomainSpec:
    """Seeded random particle velocities, affine matrices and deformation
    gradients near identity (for unit tests of the transfers and the solver)."""
    rng = np.random.default_rng(seed)
    p = spec.particles.copy()
    n, d = p.x.shape
    p.v = v_scale * rng.standard_normal((n, d))
    p.B = B_scale * rng.standard_normal((n, d, d))
    p.F = np.eye(d)[None] + F_scale * rng.standard_normal((n, d, d))
    return dataclasses.replace(spec, particles=p)


def jitter_positions(spec: DomainSpec, seed: int, frac: float = 0.2) -> DomainSpec:
    """Seeded random displacement of every particle by up to ``frac`` of a
    cell along each axis (breaks the lattice's symmetry)."""
    rng = np.random.default_rng(seed)
    p = spec.particles.copy()
    p.x = p.x + frac * spec.grid.dx * rng.uniform(-1.0, 1.0, p.x.shape)
    return dataclasses.replace(spec, particles=p)


def splitmix64(seed: int) -> Tuple[int, int]:
    """One step of the SplitMix64 generator (Steele, Lea, Flood 2014):
    returns (next_state, output)."""
    mask = (1 << 64) - 1
    state = (seed + 0x9E3779B97F4A7C15) & mask
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    z = z ^ (z >> 31)
    return state, z


def uniform3(seed: int) -> Tuple[float, float, float]:
    """Three U[0,1) draws from SplitMix64 started at ``seed`` (53-bit mantissa)."""
    out = []
    s = seed
    for _ in range(3):
        s, z = splitmix64(s)
        out.append((z >> 11) * (1.0 / (1 << 53)))
    return tuple(out)


def instance_params(i: int, scaled: bool = False):
    """(r_inc, E_inc, fine dx) of instance i of the batched inclusion family:
    r_inc = 0.03 + 0.05 u1, E_inc = 10^(7 + 2 u2), fine dx 0.01 if u3 < 0.5
    else 0.005 (literal) or 0.0025 / 0.001 (scaled), (u1, u2, u3) from
    SplitMix64 seeded 0x05AD0000 + i."""
    u1, u2, u3 = uniform3(0x05AD0000 + i)
    r_inc = 0.03 + 0.05 * u1
    E_inc = 10.0 ** (7.0 + 2.0 * u2)
    if scaled:
        dx_S = 0.0025 if u3 < 0.5 else 0.001
    else:
        dx_S = 0.01 if u3 < 0.5 else 0.005
    return r_inc, E_inc, dx_S


def inclusion_instance(i: int, scaled: bool = False, **kw):
    """Instance i of the batched inclusion family (``instance_params``)."""
    r_inc, E_inc, dx_S = instance_params(i, scaled)
    return inclusion(dx_S=dx_S, M=2, r_inc=r_inc, E_inc=E_inc, **kw)


def top_cap(x: np.ndarray, r_inc: float, center=(0.5, 0.5)) -> np.ndarray:
    """Particles of the inclusion's top cap: inside the inclusion disk and
    above its centre by more than half its radius (the objective region of
    the batched family's gradient)."""
    d = x - np.asarray(center)[None, :]
    return (np.hypot(d[:, 0], d[:, 1]) < r_inc) & (d[:, 1] > 0.5 * r_inc)


def identical_pair(spec: DomainSpec, M: int = 1):
    """Two copies of one domain (same grid, same particles, every particle a
    boundary particle) for the reduction case where every boundary node of
    one grid coincides with one of the other and the mass tie makes the
    coarse grid the donor everywhere."""
    pB = spec.particles.copy()
    pB.flags = np.full(pB.n, FLAG_BOUNDARY, np.uint8)
    pS = pB.copy()
    B = dataclasses.replace(spec, name=spec.name + "_B", particles=pB)
    S = dataclasses.replace(spec, name=spec.name + "_S", particles=pS)
    rho_m = float(pB.mass[0])
    sch = SchwarzSpec(M=M, k_max=20, eps_conv=1e-5, tau_B=rho_m, tau_S=rho_m,
                      eps_tol=1e-12 * rho_m)
    return B, S, sch
