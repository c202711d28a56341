"""FP64 CPU oracle of the OS-MPM hot path (arxiv 2605.09097).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA library is checked against.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library never
does, and nothing here imports the library.  The one module both sides share
is ``paper_2605_09097_gb300.workloads`` (seeded inputs, no method arithmetic).

What it computes (all FP64, particles kept in creation/id order):

* quadratic B-spline shape functions on a structured grid (Sec. 2.2.2,
  Eq. interpolation), APIC particle-to-grid transfer (Eq. p2g_transfer);
* the backward-Euler incremental potential E_h (Eq. discrete_energy) with the
  deformation-gradient map F_p(x_hat) (Eq. F_update) and a compressible
  neo-Hookean law, its gradient (Eq. grid_residual) and its assembled Hessian
  M/dt^2 + K;
* Newton's method with a halving backtracking line search (Sec. 2.2.5), each
  linear system solved directly (sparse LU);
* APIC grid-to-particle transfer, F update and advection (Eqs. g2p_v, g2p_B,
  F_update, advection);
* the overlapping Schwarz alternating step (Sec. 3, Alg. 1): boundary-node
  selection (Eq. boundary_grid_set), mass arbitration (Eq. overlap_donor),
  interpolation I_{B->S} (Eq. interp_BtoS), mass-weighted projection
  Pi_{S->B} (Eq. spatial_projection), temporal interpolation T_m
  (Eq. temporal_interp), interface residuals (Eqs. convergence_residuals,
  convergence_criterion) and the post-convergence coarse update (Sec. 3.5).

Readings of points the paper leaves open are stated where they are used
(shape-function order, the neo-Hookean form, the stopping rules, the boundary
layer and the coupling thresholds); the CUDA path takes the same readings.

Parity pins for every function live in ``tests/test_oracle_*.py``.  Parity
unpinned: the coupled inclusion problem under a displaced top edge has no
closed form; beyond its invariants it is checked only against the CUDA path.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2605_09097_gb300.workloads import (FLAG_BOUNDARY, DomainSpec, Dirichlet, Grid,
                                               Particles, SchwarzSpec)


class OracleError(RuntimeError):
    pass


class OutOfGrid(OracleError):
    pass


class LineSearchFailed(OracleError):
    pass


class NewtonMaxIter(OracleError):
    pass


# ----------------------------------------------------------------------------
# Shape functions (Sec. 2.2.2, Eq. interpolation).  The paper does not state
# the order; the reading is the quadratic B-spline, whose APIC inertia tensor
# is D_p = dx^2/4 I (Jiang et al., cited with Eq. p2g_transfer).
# ----------------------------------------------------------------------------

def bspline2(r: np.ndarray) -> np.ndarray:
    """Quadratic B-spline N(r) of the normalised distance r = (x - x_i)/dx:
    3/4 - r^2 for |r| < 1/2, (3/2 - |r|)^2 / 2 for 1/2 <= |r| < 3/2, else 0."""
    a = np.abs(r)
    return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))


def bspline2_deriv(r: np.ndarray) -> np.ndarray:
    """dN/dr of ``bspline2``."""
    a = np.abs(r)
    s = np.sign(r)
    return np.where(a < 0.5, -2.0 * r, np.where(a < 1.5, -s * (1.5 - a), 0.0))


def stencil_offsets(d: int) -> np.ndarray:
    """The 3^d node offsets of one particle's support, x fastest."""
    k = np.arange(3)
    return np.stack(np.meshgrid(*([k] * d), indexing="ij")[::-1], axis=-1).reshape(-1, d)


@dataclass
class Stencil:
    base: np.ndarray    # (N, d) int64, lowest node of the support
    node: np.ndarray    # (N, K) int64, flat node index (x fastest)
    nodes3: np.ndarray  # (N, K, d) int64 node multi-index
    xi: np.ndarray      # (N, K, d) node positions
    N: np.ndarray       # (N, K) weights N_i(x_p)
    dN: np.ndarray      # (N, K, d) gradients of N_i at x_p


def grid_t(x: np.ndarray, grid: Grid) -> np.ndarray:
    """(x - o) * (1/dx), the position in cell units.  The base node index is
    floor of this minus 1/2, in the same FP64 operation order on both sides
    (no fused multiply-add), so node indexing is bit-exact."""
    o = np.asarray(grid.origin, dtype=np.float64)
    inv_dx = 1.0 / grid.dx
    return (x - o[None, :]) * inv_dx


def stencil(x: np.ndarray, grid: Grid, check: bool = True) -> Stencil:
    d = grid.dim
    t = grid_t(x, grid)
    base = np.floor(t - 0.5).astype(np.int64)
    off = stencil_offsets(d)
    nodes3 = base[:, None, :] + off[None, :, :]
    res = np.asarray(grid.res)
    if check and (np.any(nodes3 < 0) or np.any(nodes3 >= res[None, None, :])):
        raise OutOfGrid("a particle's support leaves the grid box")
    o = np.asarray(grid.origin, dtype=np.float64)
    xi = o[None, None, :] + nodes3 * grid.dx
    r = t[:, None, :] - nodes3          # (N, K, d) normalised distances
    w = bspline2(r)
    dw = bspline2_deriv(r) / grid.dx
    N = np.prod(w, axis=2)
    dN = np.empty_like(r)
    for a in range(d):
        others = [b for b in range(d) if b != a]
        dN[:, :, a] = dw[:, :, a] * np.prod(w[:, :, others], axis=2)
    flat = np.zeros(nodes3.shape[:2], dtype=np.int64)
    stride = 1
    for a in range(d):
        flat += nodes3[:, :, a] * stride
        stride *= int(res[a])
    return Stencil(base, flat, nodes3, xi, N, dN)


def node_positions(grid: Grid) -> np.ndarray:
    """Positions of all grid nodes, (n_nodes, d), x fastest."""
    axes = [grid.origin[a] + np.arange(grid.res[a]) * grid.dx for a in range(grid.dim)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    return np.stack([m.reshape(-1) for m in mesh], axis=-1)


# ----------------------------------------------------------------------------
# Morton order of the particles (not in the paper; the CUDA path keeps its
# particles sorted by the Morton code of their base node, ties by id).
# ----------------------------------------------------------------------------

def morton_code(base: np.ndarray, bits: int = 21) -> np.ndarray:
    """Interleave the bits of the base-node multi-index, axis 0 in the least
    significant position (bit by bit, brute force)."""
    n, d = base.shape
    code = np.zeros(n, dtype=np.uint64)
    b = base.astype(np.uint64)
    for bit in range(bits):
        for a in range(d):
            code |= ((b[:, a] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(bit * d + a)
    return code


def sort_order(x: np.ndarray, grid: Grid) -> np.ndarray:
    """Particle ids in Morton order (stable: equal codes keep id order)."""
    st = stencil(x, grid)
    return np.argsort(morton_code(st.base), kind="stable")


# ----------------------------------------------------------------------------
# Constitutive law.  The paper names a neo-Hookean solid (Sec. 4) without its
# form; the reading is the compressible model
#   Psi = mu/2 (tr F^T F - d) - mu ln J + lam/2 (ln J)^2,
# mu = E / (2(1+nu)), lam = E nu / ((1+nu)(1-2nu)) (plane strain in 2D, as the
# Lame formulas of Sec. 4.3 assume).  J <= 0 gives Psi = +inf.
# ----------------------------------------------------------------------------

def lame(E: np.ndarray, nu: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def _det_minus_one(H: np.ndarray) -> np.ndarray:
    """det(I + H) - 1 expanded in H (no cancellation for small H):
    2D: tr H + det H; 3D: tr H + (sum of principal 2x2 minors) + det H."""
    d = H.shape[-1]
    tr = np.trace(H, axis1=1, axis2=2)
    if d == 2:
        return tr + (H[:, 0, 0] * H[:, 1, 1] - H[:, 0, 1] * H[:, 1, 0])
    m2 = (H[:, 0, 0] * H[:, 1, 1] - H[:, 0, 1] * H[:, 1, 0]
          + H[:, 0, 0] * H[:, 2, 2] - H[:, 0, 2] * H[:, 2, 0]
          + H[:, 1, 1] * H[:, 2, 2] - H[:, 1, 2] * H[:, 2, 1])
    return tr + m2 + np.linalg.det(H)


def psi(F: np.ndarray, mu: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Psi(F) per particle.  Evaluated through H = F - I (exact in FP64 for
    F near I) as mu/2 (2 tr H + |H|^2) - mu ln J + lam/2 (ln J)^2 with
    ln J = log1p(det(I+H) - 1), so small strains do not cancel."""
    d = F.shape[-1]
    H = F - np.eye(d)[None]
    jm1 = _det_minus_one(H)
    out = np.full(jm1.shape, np.inf)
    ok = jm1 > -1.0
    lnJ = np.log1p(jm1[ok])
    Hk = H[ok]
    I1md = 2.0 * np.trace(Hk, axis1=1, axis2=2) + np.sum(Hk ** 2, axis=(1, 2))
    out[ok] = 0.5 * mu[ok] * I1md - mu[ok] * lnJ + 0.5 * lam[ok] * lnJ ** 2
    return out


def _det_change(F0: np.ndarray, dF: np.ndarray) -> np.ndarray:
    """det(F0 + dF) - det(F0) as a polynomial in dF (exact identity):
    2D: F0_00 dF_11 + dF_00 F0_11 + det dF - F0_01 dF_10 - dF_01 F0_10;
    3D: cof(F0):dF + F0:cof(dF) + det dF."""
    d = F0.shape[-1]
    if d == 2:
        return (F0[:, 0, 0] * dF[:, 1, 1] + dF[:, 0, 0] * F0[:, 1, 1]
                - F0[:, 0, 1] * dF[:, 1, 0] - dF[:, 0, 1] * F0[:, 1, 0]
                + dF[:, 0, 0] * dF[:, 1, 1] - dF[:, 0, 1] * dF[:, 1, 0])

    def cof(A):
        return np.stack([np.cross(A[:, 1], A[:, 2]), np.cross(A[:, 2], A[:, 0]),
                         np.cross(A[:, 0], A[:, 1])], axis=1)
    return (np.sum(cof(F0) * dF, axis=(1, 2)) + np.sum(F0 * cof(dF), axis=(1, 2))
            + np.linalg.det(dF))


def psi_change(F0: np.ndarray, dF: np.ndarray, mu: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Psi(F0 + dF) - Psi(F0) per particle, through exact difference
    identities: mu (F0:dF + |dF|^2/2) - mu dl + lam/2 dl (2 ln J0 + dl) with
    dl = ln J1 - ln J0 = log1p(dJ / J0).  Its rounding error scales with dF,
    not with F (the line search of Sec. 2.2.5 compares changes down to the
    Newton tolerance).  +inf where J0 + dJ <= 0."""
    d = F0.shape[-1]
    jm1 = _det_minus_one(F0 - np.eye(d)[None])
    J0 = 1.0 + jm1
    dJ = _det_change(F0, dF)
    out = np.full(J0.shape, np.inf)
    ok = (J0 > 0) & (J0 + dJ > 0)
    dl = np.log1p(dJ[ok] / J0[ok])
    lnJ0 = np.log1p(jm1[ok])
    m, l = mu[ok], lam[ok]
    out[ok] = (m * (np.sum(F0[ok] * dF[ok], axis=(1, 2)) + 0.5 * np.sum(dF[ok] ** 2, axis=(1, 2)))
               - m * dl + 0.5 * l * dl * (2.0 * lnJ0 + dl))
    return out


def pk1(F: np.ndarray, mu: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """First Piola-Kirchhoff stress dPsi/dF = mu (F - F^-T) + lam ln J F^-T."""
    J = np.linalg.det(F)
    if np.any(J <= 0):
        raise OracleError("inverted element (J <= 0) in the stress evaluation")
    FinvT = np.transpose(np.linalg.inv(F), (0, 2, 1))
    return mu[:, None, None] * (F - FinvT) + (lam * np.log(J))[:, None, None] * FinvT


def cauchy_stress(F: np.ndarray, mu: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """sigma = P F^T / J (the Cauchy stress of ``pk1``)."""
    J = np.linalg.det(F)
    return np.einsum("pab,pcb->pac", pk1(F, mu, lam), F) / J[:, None, None]


def dpdf(F: np.ndarray, mu: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Fourth-order tangent A[p, a, c, b, e] = dP_ac / dF_be of ``pk1``:
    mu d_ab d_ce + (mu - lam ln J) Finv_ea Finv_cb + lam Finv_ca Finv_eb."""
    n, d, _ = F.shape
    J = np.linalg.det(F)
    Finv = np.linalg.inv(F)
    I = np.eye(d)
    A = mu[:, None, None, None, None] * np.einsum("ab,ce->acbe", I, I)[None]
    A = A + ((mu - lam * np.log(J))[:, None, None, None, None]
             * np.einsum("pea,pcb->pacbe", Finv, Finv))
    A = A + lam[:, None, None, None, None] * np.einsum("pca,peb->pacbe", Finv, Finv)
    return A


# ----------------------------------------------------------------------------
# Transfers (Sec. 2.2.4)
# ----------------------------------------------------------------------------

@dataclass
class GridFields:
    m: np.ndarray        # (nn,) nodal mass
    mv: np.ndarray       # (nn, d) nodal momentum
    vn: np.ndarray       # (nn, d) v^n = mv / m on active nodes, 0 elsewhere
    active: np.ndarray   # (nn,) bool, m > 0
    bm: Optional[np.ndarray] = None  # (nn,) boundary-particle mass (Eq. boundary_grid_set)


def p2g(p: Particles, grid: Grid, boundary_mass: bool = False, mass_eps: float = 0.0) -> GridFields:
    """APIC particle-to-grid transfer, Eq. p2g_transfer (and Eq. p2g_substep):
    m_i = sum_p m_p N_i(x_p), (mv)_i = sum_p m_p N_i (v_p + B_p D_p^-1 (x_i - x_p)),
    D_p^-1 = 4/dx^2 I for the quadratic B-spline.  With ``boundary_mass`` also
    returns sum over boundary particles of m_p N_i (Eq. boundary_grid_set).
    The active node set (N_alpha of Sec. 3.2.1) is m_i > mass_eps: nodes that
    a particle touches only with a round-off-sized weight carry no DOF."""
    d = grid.dim
    nn = grid.n_nodes
    st = stencil(p.x, grid)
    Dinv = 4.0 / grid.dx ** 2
    m = np.zeros(nn)
    np.add.at(m, st.node, p.mass[:, None] * st.N)
    dxp = st.xi - p.x[:, None, :]                          # x_i - x_p
    vel = p.v[:, None, :] + Dinv * np.einsum("pab,pkb->pka", p.B, dxp)
    mv = np.zeros((nn, d))
    for a in range(d):
        np.add.at(mv[:, a], st.node, p.mass[:, None] * st.N * vel[:, :, a])
    active = m > mass_eps
    vn = np.zeros((nn, d))
    vn[active] = mv[active] / m[active, None]
    bm = None
    if boundary_mass:
        isb = (p.flags & FLAG_BOUNDARY) != 0
        bm = np.zeros(nn)
        np.add.at(bm, st.node[isb], p.mass[isb, None] * st.N[isb])
    return GridFields(m, mv, vn, active, bm)


def deformation(p: Particles, st: Stencil, u: np.ndarray) -> np.ndarray:
    """Eq. F_update: F_p(x_hat) = (I + sum_i (x_hat_i - x_i^n) grad N_i(x_p)^T) F_p^n,
    with u_i = x_hat_i - x_i^n."""
    d = p.x.shape[1]
    G = np.einsum("pka,pkb->pab", u[st.node], st.dN)
    return np.einsum("pab,pbc->pac", np.eye(d)[None] + G, p.F)


def g2p(p: Particles, grid: Grid, u: np.ndarray, dt: float) -> Particles:
    """APIC grid-to-particle transfer with v_i^{n+1} = u_i / dt (Eqs. g2p_v,
    g2p_B), the deformation-gradient update (Eq. F_update, equivalently
    Eq. F_substep) and advection (Eq. advection).  Returns new particles."""
    st = stencil(p.x, grid)
    vgrid = u / dt
    vk = vgrid[st.node]                                     # (N, K, d)
    v_new = np.einsum("pk,pka->pa", st.N, vk)
    B_new = np.einsum("pk,pka,pkb->pab", st.N, vk, st.xi - p.x[:, None, :])
    F_new = deformation(p, st, u)
    q = p.copy()
    q.v = v_new
    q.B = B_new
    q.F = F_new
    q.x = p.x + dt * v_new
    return q


# ----------------------------------------------------------------------------
# Dirichlet data
# ----------------------------------------------------------------------------

def rotation_matrix(axis: Sequence[float], angle: float, d: int) -> np.ndarray:
    """Rodrigues' rotation by ``angle`` about the unit ``axis`` (2D: about z)."""
    if d == 2:
        c, s = np.cos(angle), np.sin(angle)
        return np.array([[c, -s], [s, c]])
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(angle) * Kx + (1 - np.cos(angle)) * (Kx @ Kx)


def dirichlet_nodes(grid: Grid, rules: Sequence[Dirichlet], dt: float):
    """Node-wise prescribed velocities: returns (mask (nn, d) bool, vel (nn, d)).
    A node is in a rule when lo <= x_i <= hi on every axis; later rules
    override earlier ones on the components they set."""
    d = grid.dim
    xi = node_positions(grid)
    nn = xi.shape[0]
    mask = np.zeros((nn, d), dtype=bool)
    vel = np.zeros((nn, d))
    for r in rules:
        lo = np.asarray(r.lo[:d])
        hi = np.asarray(r.hi[:d])
        inside = np.all((xi >= lo[None]) & (xi <= hi[None]), axis=1)
        if r.kind == 0:
            for a in range(d):
                if (r.comp_mask >> a) & 1:
                    mask[inside, a] = True
                    vel[inside, a] = r.vel[a]
        elif r.kind == 1:
            R = rotation_matrix(r.axis, r.omega * dt, d)
            c = np.asarray(r.center[:d])
            rel = xi[inside] - c[None]
            vel[inside] = (rel @ R.T - rel) / dt
            mask[inside] = True
        else:
            raise OracleError(f"unknown Dirichlet kind {r.kind}")
    return mask, vel


# ----------------------------------------------------------------------------
# Incremental potential and Newton (Sec. 2.2.3, 2.2.5)
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """One backward-Euler step of one domain, parameterised by the grid
    displacement u_i = x_hat_i - x_i^n (Sec. 2.2.3)."""
    p: Particles
    grid: Grid
    dt: float
    gf: GridFields
    st: Stencil
    mu: np.ndarray
    lam: np.ndarray
    fext: np.ndarray      # (nn, d) = m_i g (Eq. f_ext; no traction)
    fixed: np.ndarray     # (nn, d) bool: Dirichlet DOFs (inactive nodes are fixed at 0 too)
    u_fixed: np.ndarray   # (nn, d) prescribed displacement on fixed DOFs

    @property
    def free(self) -> np.ndarray:
        return self.gf.active[:, None] & ~self.fixed


def make_problem(p: Particles, grid: Grid, gf: GridFields, dt: float,
                 gravity: Sequence[float], mask: np.ndarray, vel: np.ndarray) -> Problem:
    d = grid.dim
    st = stencil(p.x, grid)
    mu, lam = lame(p.E, p.nu)
    g = np.asarray(gravity[:d], dtype=np.float64)
    fext = gf.m[:, None] * g[None, :]
    fixed = mask & gf.active[:, None]
    u_fixed = np.where(fixed, dt * vel, 0.0)
    return Problem(p, grid, dt, gf, st, mu, lam, fext, fixed, u_fixed)


def initial_guess(pr: Problem) -> np.ndarray:
    """Newton's starting iterate (reading: the paper does not fix it): on the
    free DOFs x_tilde = x^n + dt v^n, or x^n itself when that has the strictly
    lower E_h (E_h(x_tilde) - E_h(x^n) > 0, +inf when x_tilde inverts an
    element); the prescribed value on Dirichlet DOFs and 0 on inactive nodes
    either way.  Under large quasi-static steps (dt far above the slowest
    period, Sec. 2.2.6) x_tilde extrapolates a transient the step removes and
    x^n is the better start; for resolved dynamics x_tilde wins."""
    u_n = np.where(pr.fixed, pr.u_fixed, 0.0)
    u = np.where(pr.gf.active[:, None], pr.dt * pr.gf.vn, 0.0)
    u_tilde = np.where(pr.fixed, pr.u_fixed, u)
    if energy_change(pr, u_n, u_tilde - u_n, 1.0) > 0.0:
        return u_n
    return u_tilde


def energy(pr: Problem, u: np.ndarray) -> float:
    """Eq. discrete_energy in u: sum_i m_i/(2dt^2)|u_i - dt v_i^n|^2
    + sum_p V_p^0 Psi(F_p(u)) - sum_i u_i . f_i^ext.  The constant
    -sum_i x_i^n . f_i^ext is dropped (the line search compares values only)."""
    a = pr.gf.active
    inert = np.sum(pr.gf.m[a, None] / (2.0 * pr.dt ** 2) * (u[a] - pr.dt * pr.gf.vn[a]) ** 2)
    F = deformation(pr.p, pr.st, u)
    el = np.sum(pr.p.vol0 * psi(F, pr.mu, pr.lam))
    return float(inert + el - np.sum(u[a] * pr.fext[a]))


def energy_change(pr: Problem, u: np.ndarray, step: np.ndarray, alpha: float) -> float:
    """E_h(u + alpha step) - E_h(u), summed term by term: per node
    m_i/(2dt^2) (alpha s_i).(2(u_i - dt v_i^n) + alpha s_i) - alpha s_i . f_i,
    per particle V_p^0 (Psi(F_p(u) + dF_p) - Psi(F_p(u))) with
    dF_p = alpha (sum_i s_i grad N_i^T) F_p^n (``psi_change``).  Equal to the
    difference of two ``energy`` values, without the cancellation of the
    large terms they hold (the line-search test of Sec. 2.2.5 is the sign of
    this number).  +inf when a trial inverts an element."""
    a = pr.gf.active
    s = alpha * step
    inert = np.sum(pr.gf.m[a, None] / (2.0 * pr.dt ** 2)
                   * s[a] * (2.0 * (u[a] - pr.dt * pr.gf.vn[a]) + s[a]))
    ext = -np.sum(s[a] * pr.fext[a])
    F0 = deformation(pr.p, pr.st, u)
    Gs = np.einsum("pka,pkb->pab", s[pr.st.node], pr.st.dN)
    dF = np.einsum("pab,pbc->pac", Gs, pr.p.F)
    dpsi = psi_change(F0, dF, pr.mu, pr.lam)
    if not np.all(np.isfinite(dpsi)):
        return float("inf")
    return float(inert + ext + np.sum(pr.p.vol0 * dpsi))


def gradient(pr: Problem, u: np.ndarray) -> np.ndarray:
    """dE_h/du_i = m_i/dt^2 (u_i - dt v_i^n) + sum_p V_p^0 P_p F_p^{nT} grad N_i
    - f_i^ext (Eq. grid_residual with the energy-consistent internal force)."""
    nn, d = u.shape
    F = deformation(pr.p, pr.st, u)
    P = pk1(F, pr.mu, pr.lam)
    C = np.einsum("pba,pkb->pka", pr.p.F, pr.st.dN)        # F^{nT} grad N_i
    fint = pr.p.vol0[:, None, None] * np.einsum("pab,pkb->pka", P, C)
    g = pr.gf.m[:, None] / pr.dt ** 2 * (u - pr.dt * pr.gf.vn) - pr.fext
    for a in range(d):
        np.add.at(g[:, a], pr.st.node, fint[:, :, a])
    return np.where(pr.gf.active[:, None], g, 0.0)


def hessian(pr: Problem, u: np.ndarray) -> sp.csr_matrix:
    """M/dt^2 + K with K the Hessian of sum_p V_p^0 Psi(F_p(u)) (Sec. 2.2.5),
    assembled over all (node, component) DOFs, index node*d + component."""
    nn, d = u.shape
    F = deformation(pr.p, pr.st, u)
    A = dpdf(F, pr.mu, pr.lam)
    C = np.einsum("pba,pkb->pka", pr.p.F, pr.st.dN)
    Kloc = pr.p.vol0[:, None, None, None, None] * np.einsum("pkc,pacbe,ple->pkalb", C, A, C, optimize=True)
    Np, K = pr.st.node.shape
    dof = pr.st.node[:, :, None] * d + np.arange(d)[None, None, :]     # (N, K, d)
    rows = np.broadcast_to(dof[:, :, :, None, None], (Np, K, d, K, d))
    cols = np.broadcast_to(dof[:, None, None, :, :], (Np, K, d, K, d))
    H = sp.coo_matrix((Kloc.reshape(-1), (rows.reshape(-1), cols.reshape(-1))),
                      shape=(nn * d, nn * d)).tocsr()
    mdiag = np.repeat(pr.gf.m / pr.dt ** 2, d)
    return (H + sp.diags(mdiag)).tocsr()


@dataclass
class NewtonStats:
    iters: int = 0
    ls_halvings: int = 0


def newton(pr: Problem, newton_tol: float, newton_max: int, ls_max: int,
           stats: Optional[NewtonStats] = None) -> np.ndarray:
    """Newton's method with backtracking line search (Sec. 2.2.5).  Stop
    when max |delta| / dt <= newton_tol on the free DOFs, tested before the
    line search and with the full step applied; otherwise alpha = 1, 1/2, ...
    down to 2^-ls_max until E_h strictly decreases (``energy_change`` < 0)."""
    u = initial_guess(pr)
    free = pr.free.reshape(-1)
    idx = np.nonzero(free)[0]
    st = stats if stats is not None else NewtonStats()
    for it in range(newton_max):
        st.iters = it + 1
        if idx.size == 0:
            return u
        g = gradient(pr, u).reshape(-1)[idx]
        H = hessian(pr, u)[idx][:, idx]
        delta = spla.spsolve(H.tocsc(), -g)
        if np.dot(delta, g) >= 0.0 and np.any(g != 0.0):
            delta = -g
        step = np.zeros(u.size)
        step[idx] = delta
        step = step.reshape(u.shape)
        if np.max(np.abs(delta)) <= newton_tol * pr.dt:
            return u + step
        alpha = 1.0
        for s in range(ls_max + 1):
            if energy_change(pr, u, step, alpha) < 0.0:
                break
            alpha *= 0.5
            st.ls_halvings += 1
        else:
            raise LineSearchFailed("no decrease of E_h after the halving cap")
        u = u + alpha * step
    raise NewtonMaxIter("Newton did not reach its tolerance")


# ----------------------------------------------------------------------------
# Single-domain step
# ----------------------------------------------------------------------------

@dataclass
class DomainState:
    spec: DomainSpec
    p: Particles

    @classmethod
    def create(cls, spec: DomainSpec) -> "DomainState":
        return cls(spec, spec.particles.copy())


def solve_domain(ds: DomainState, gf: GridFields, dt: float,
                 extra_mask: Optional[np.ndarray] = None,
                 extra_vel: Optional[np.ndarray] = None,
                 stats: Optional[NewtonStats] = None) -> np.ndarray:
    """Implicit solve of one domain for dt with its physical Dirichlet rules
    plus (optionally) Schwarz receiver nodes; physical rules win."""
    spec = ds.spec
    mask, vel = dirichlet_nodes(spec.grid, spec.dirichlet, dt)
    if extra_mask is not None:
        add = extra_mask[:, None] & ~mask
        vel = np.where(add, extra_vel, vel)
        mask = mask | add
    pr = make_problem(ds.p, spec.grid, gf, dt, spec.gravity, mask, vel)
    return newton(pr, spec.newton_tol, spec.newton_max, spec.ls_max, stats)


def step(ds: DomainState, dt: float, stats: Optional[NewtonStats] = None) -> np.ndarray:
    """One backward-Euler MPM step of a single domain: P2G, Newton solve,
    G2P with F update and advection.  Returns the solved grid displacement."""
    gf = p2g(ds.p, ds.spec.grid, mass_eps=ds.spec.mass_eps)
    u = solve_domain(ds, gf, dt, stats=stats)
    ds.p = g2p(ds.p, ds.spec.grid, u, dt)
    return u


# ----------------------------------------------------------------------------
# Interface operators (Sec. 3.2)
# ----------------------------------------------------------------------------

def boundary_sets(gf: GridFields, tau: float) -> np.ndarray:
    """Eq. boundary_grid_set: active nodes whose boundary-particle mass
    exceeds tau_Gamma."""
    return gf.active & (gf.bm > tau)


def coincident_fine_node(gB: Grid, gS: Grid) -> np.ndarray:
    """For each coarse node, the flat index of the fine node at the same
    place (|x_B - x_S|_inf <= 1e-9 dx_S), or -1."""
    xB = node_positions(gB)
    oS = np.asarray(gS.origin)
    j3 = np.rint((xB - oS[None]) / gS.dx).astype(np.int64)
    resS = np.asarray(gS.res)
    inside = np.all((j3 >= 0) & (j3 < resS[None]), axis=1)
    xS = oS[None] + j3 * gS.dx
    close = np.all(np.abs(xS - xB) <= 1e-9 * gS.dx, axis=1)
    flat = np.zeros(len(xB), dtype=np.int64)
    stride = 1
    for a in range(gS.dim):
        flat += j3[:, a] * stride
        stride *= int(resS[a])
    return np.where(inside & close, flat, -1)


def projection_sums(gB: Grid, gS: Grid, mS: np.ndarray, vS: np.ndarray,
                    activeS: np.ndarray):
    """Numerator and denominator of Eq. spatial_projection over the whole
    coarse grid: sum_j m_Sj v_Sj N_BI(x_Sj) and sum_j m_Sj N_BI(x_Sj) over
    active fine nodes j.  Support nodes outside the coarse box are dropped."""
    d = gB.dim
    xS = node_positions(gS)[activeS]
    st = stencil(xS, gB, check=False)
    res = np.asarray(gB.res)
    ok = np.all((st.nodes3 >= 0) & (st.nodes3 < res[None, None]), axis=2)
    w = mS[activeS][:, None] * st.N * ok
    node = np.where(ok, st.node, 0)
    den = np.zeros(gB.n_nodes)
    np.add.at(den, node, w)
    num = np.zeros((gB.n_nodes, d))
    for a in range(d):
        np.add.at(num[:, a], node, w * vS[activeS][:, a][:, None])
    return num, den


def project_S2B(gB: Grid, gS: Grid, gfS: GridFields, recvB: np.ndarray, eps_tol: float) -> np.ndarray:
    """Pi_{S->B} (Eq. spatial_projection) on the coarse receiver nodes;
    (nB, d) with zeros off the receiver set."""
    num, den = projection_sums(gB, gS, gfS.m, gfS.vn, gfS.active)
    out = np.zeros_like(num)
    out[recvB] = num[recvB] / (den[recvB, None] + eps_tol)
    return out


def substep_average(grids: Sequence[GridFields], vels: Sequence[np.ndarray]) -> GridFields:
    """Time average over one coarse step of the fine sub-steps' solved grids:
    mass (1/M) sum_m m^(m) and momentum (1/M) sum_m m^(m) v^(m), each sub-step
    over its own active nodes.  Reading of v_S^(k) in Eq. implicit_solve_coarse:
    the coarse solve prescribes a velocity held over the whole step dT, like
    v_B = (x_B - x_B^n)/dT, so the fine side supplies its motion over the same
    interval, not its velocity at the last sub-step.  With M = 1 it is the
    solved fine grid of the single sub-step."""
    M = len(grids)
    m = np.zeros_like(grids[0].m)
    mv = np.zeros_like(grids[0].mv)
    for gf, v in zip(grids, vels):
        a = gf.active
        m[a] += gf.m[a] / M
        mv[a] += gf.m[a, None] * v[a] / M
    active = m > 0.0
    vn = np.zeros_like(mv)
    vn[active] = mv[active] / m[active, None]
    return GridFields(m, mv, vn, active)


def interp_B2S(gB: Grid, gS: Grid, vB: np.ndarray, recvS: np.ndarray) -> np.ndarray:
    """I_{B->S} (Eq. interp_BtoS) on the fine receiver nodes: sum over the
    coarse support of v_BI N_BI(x_Sj); (nS, d) with zeros off the set."""
    d = gB.dim
    out = np.zeros((gS.n_nodes, d))
    idx = np.nonzero(recvS)[0]
    if idx.size == 0:
        return out
    xS = node_positions(gS)[idx]
    st = stencil(xS, gB)
    out[idx] = np.einsum("pk,pka->pa", st.N, vB[st.node])
    return out


def coarse_support_active(gB: Grid, gS: Grid, activeB: np.ndarray) -> np.ndarray:
    """For each fine node: are all coarse support nodes inside the box and active?"""
    xS = node_positions(gS)
    st = stencil(xS, gB, check=False)
    res = np.asarray(gB.res)
    ok = np.all((st.nodes3 >= 0) & (st.nodes3 < res[None, None]), axis=2)
    node = np.where(ok, st.node, 0)
    return np.all(ok & activeB[node], axis=1)


@dataclass
class InterfaceSets:
    recvB: np.ndarray   # (nB,) bool, Gamma_hat_B
    recvS: np.ndarray   # (nS,) bool, Gamma_hat_S
    gammaB: np.ndarray  # (nB,) bool, Gamma_B before arbitration
    gammaS: np.ndarray  # (nS,) bool


def interface_sets(B: DomainState, S: DomainState, gfB: GridFields, gfS: GridFields,
                   sch: SchwarzSpec, dT: float) -> InterfaceSets:
    """Boundary sets (Eq. boundary_grid_set) and overlap arbitration
    (Eq. overlap_donor).  Readings: a coincident pair of boundary nodes is
    donated by the larger grid mass, with ties (within 1e-12 relative) going
    to B; Gamma_hat_B keeps nodes with fine projection mass > tau_B;
    Gamma_hat_S keeps nodes whose coarse support is all active; nodes with a
    physical Dirichlet rule never receive."""
    gB, gS = B.spec.grid, S.spec.grid
    gamB = boundary_sets(gfB, sch.tau_B)
    gamS = boundary_sets(gfS, sch.tau_S)
    recvB = gamB.copy()
    recvS = gamS.copy()
    j = coincident_fine_node(gB, gS)
    for I in np.nonzero(gamB & (j >= 0))[0]:
        jj = j[I]
        if not gamS[jj]:
            continue
        mB, mS = gfB.m[I], gfS.m[jj]
        if mS > mB * (1.0 + 1e-12):      # S donates, B receives
            recvS[jj] = False
        else:                             # B donates (ties to B), S receives
            recvB[I] = False
    _, den = projection_sums(gB, gS, gfS.m, gfS.vn, gfS.active)
    recvB &= den > sch.tau_B
    recvS &= coarse_support_active(gB, gS, gfB.active)
    mB, _ = dirichlet_nodes(gB, B.spec.dirichlet, dT)
    mS, _ = dirichlet_nodes(gS, S.spec.dirichlet, dT / sch.M)
    recvB &= ~np.any(mB, axis=1)
    recvS &= ~np.any(mS, axis=1)
    return InterfaceSets(recvB, recvS, gamB, gamS)


def time_interp(v0: np.ndarray, v1: np.ndarray, m: int, M: int) -> np.ndarray:
    """T_m of Eq. temporal_interp: (1 - m/M) v^n + (m/M) v^{n+1}."""
    a = m / M
    return (1.0 - a) * v0 + a * v1


def rel_change(new: np.ndarray, old: np.ndarray, mask: np.ndarray) -> float:
    """One of Eq. convergence_residuals over the receiver set: |new - old|_2 /
    |new|_2, or the absolute norm when |new|_2 < 1e-14 or the set is empty."""
    num = float(np.sqrt(np.sum((new[mask] - old[mask]) ** 2)))
    den = float(np.sqrt(np.sum(new[mask] ** 2)))
    return num if den < 1e-14 else num / den


@dataclass
class SchwarzStats:
    iters: int = 0
    r_B: float = 0.0
    r_S: float = 0.0
    converged: bool = False
    history: List[Tuple[float, float]] = field(default_factory=list)
    newton_B: List[int] = field(default_factory=list)
    newton_S: List[int] = field(default_factory=list)


def schwarz_step(B: DomainState, S: DomainState, dT: float, sch: SchwarzSpec,
                 stats: Optional[SchwarzStats] = None,
                 sets_out: Optional[dict] = None) -> None:
    """One global step of the alternating Schwarz method, Alg. 1.

    Readings: the coarse BC of iteration k >= 1 is Pi of the fine grid
    velocity of iteration k-1 averaged over its M sub-steps (substep_average;
    with ``sch.pi_source == 1`` the P2G grid that ends sub-step M instead;
    for k = 0, Pi of the fine P2G at t_n); v_B^(0) is the coarse P2G velocity at t_n; convergence needs
    k >= 1; k runs 0..k_max.  P_S is not reset after convergence; P_B takes
    one G2P + advection with the last coarse solution (Sec. 3.5)."""
    st = stats if stats is not None else SchwarzStats()
    M = sch.M
    dt = dT / M
    gB, gS = B.spec.grid, S.spec.grid
    # Step 0 (Eq. store_states): snapshot of the fine particles
    snap = S.p.copy()
    gfB = p2g(B.p, gB, boundary_mass=True, mass_eps=B.spec.mass_eps)
    gfS = p2g(S.p, gS, boundary_mass=True, mass_eps=S.spec.mass_eps)
    sets = interface_sets(B, S, gfB, gfS, sch, dT)
    if sets_out is not None:
        sets_out["sets"] = sets
        sets_out["gfB"] = gfB
        sets_out["gfS"] = gfS
    vGB = project_S2B(gB, gS, gfS, sets.recvB, sch.eps_tol)    # v_GammaB^(0)
    vGS = interp_B2S(gB, gS, gfB.vn, sets.recvS)                # I(v_B^(0) = v_B^n)
    vSn = vGS.copy()                                            # I(v_B^n), fixed in the frame
    uB = None
    for k in range(sch.k_max + 1):
        # 1. coarse solve with Pi BCs (Eq. implicit_solve_coarse)
        ns = NewtonStats()
        uB = solve_domain(B, gfB, dT, sets.recvB, vGB, ns)
        st.newton_B.append(ns.iters)
        vB_new = np.where(gfB.active[:, None], uB / dT, 0.0)
        # 2. fine sub-cycling (Eqs. spatial_interp_n, implicit_solve_fine)
        S.p = snap.copy()
        gf = p2g(S.p, gS, mass_eps=S.spec.mass_eps)
        vSnp1 = interp_B2S(gB, gS, vB_new, sets.recvS)
        solved, vels = [], []
        for m in range(1, M + 1):
            bc = time_interp(vSn, vSnp1, m, M)
            ns = NewtonStats()
            uS = solve_domain(S, gf, dt, sets.recvS, bc, ns)
            st.newton_S.append(ns.iters)
            solved.append(gf)
            vels.append(uS / dt)
            S.p = g2p(S.p, gS, uS, dt)
            gf = p2g(S.p, gS, mass_eps=S.spec.mass_eps)
        # 3. convergence (Eqs. convergence_residuals, convergence_criterion)
        src = substep_average(solved, vels) if sch.pi_source == 0 else gf
        vGB_new = project_S2B(gB, gS, src, sets.recvB, sch.eps_tol)
        rB = rel_change(vGB_new, vGB, sets.recvB)
        rS = rel_change(vSnp1, vGS, sets.recvS)
        st.history.append((rB, rS))
        st.iters = k + 1
        st.r_B, st.r_S = rB, rS
        vGB, vGS = vGB_new, vSnp1
        if k >= 1 and rB <= sch.eps_conv and rS <= sch.eps_conv:
            st.converged = True
            break
    # 4. post-convergence coarse update (Sec. 3.5)
    B.p = g2p(B.p, gB, uB, dT)
