"""Reverse-mode gradients through backward-Euler MPM steps (Sec. 2.2).

TEST INFRASTRUCTURE ONLY.  This is the slow, plain reference for the CUDA
library's adjoint: only the tests may import it; the library never does, and
nothing here imports the library.

A step maps the particle state s^n = (x, v, B, F) and the Young's moduli E to
s^{n+1} through three stages:

* P2G (Eq. p2g_transfer): m_i = sum_p m_p N_ip, q_i = sum_p m_p N_ip (v_p +
  B_p D_p^-1 (x_i - x_p)), v_i = q_i / m_i on the active nodes;
* the implicit solve (Sec. 2.2.5): u* with g(u*) = 0 on the free DOFs,
  g_i = m_i/dt^2 (u_i - dt v_i) - m_i g_ext + sum_p V_p P(F_p(u)) F_p^T grad N_ip,
  F_p(u) = (I + sum_i u_i grad N_ip^T) F_p;
* G2P with the F update and advection (Eqs. g2p_v, g2p_B, F_update,
  advection): x' = x + sum_i N_ip u_i, v' = sum_i N_ip u_i / dt,
  B' = sum_i N_ip u_i/dt (x_i - x_p)^T, F' = F_p(u*).

The adjoint of the solve is the implicit function theorem: with
K = dg/du (the Newton Hessian M/dt^2 + K, symmetric) restricted to the free
DOFs, K lam = u_bar and z_bar -= lam . dg/dz for every input z of g.  The
active node set and the Dirichlet DOFs are held fixed (they change only at
isolated states).  N_ip depends on x_p, so the position adjoints carry
grad N and the B-spline Hessian d2N/dx2.  The Newton system is solved
exactly (sparse LU).

Pins: ``tests/test_oracle_adjoint.py`` checks every adjoint against central
finite differences of the oracle's forward step.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import scipy.sparse.linalg as spla

from oracle import osmpm_oracle as O


def bspline2_second(r: np.ndarray) -> np.ndarray:
    """d2N/dr2 of the quadratic B-spline: -2 for |r| < 1/2, 1 for
    1/2 <= |r| < 3/2, 0 outside (its value at the breakpoints is one of the
    one-sided limits; the forward map is C^1 there)."""
    a = np.abs(r)
    return np.where(a < 0.5, -2.0, np.where(a < 1.5, 1.0, 0.0))


def stencil_hessian(x: np.ndarray, grid, st: O.Stencil) -> np.ndarray:
    """(N, K, d, d): the Hessian of N_i(x) at x = x_p for every stencil node."""
    d = grid.dim
    t = O.grid_t(x, grid)
    r = t[:, None, :] - st.nodes3
    w = O.bspline2(r)
    dw = O.bspline2_deriv(r) / grid.dx
    ddw = bspline2_second(r) / grid.dx ** 2
    n, K = st.N.shape
    H = np.empty((n, K, d, d))
    for a in range(d):
        for b in range(d):
            f = np.ones((n, K))
            for c in range(d):
                if a == b:
                    f = f * (ddw[:, :, c] if c == a else w[:, :, c])
                else:
                    f = f * (dw[:, :, c] if c in (a, b) else w[:, :, c])
            H[:, :, a, b] = f
    return H


@dataclass
class StepRecord:
    """What one forward step needs kept for its adjoint."""
    p: O.Particles          # state at t_n
    pr: O.Problem           # P2G grid, stencil, masks at t_n
    u: np.ndarray           # converged grid displacement (nn, d)


def record_step(ds: O.DomainState, dt: float, newton_tol: Optional[float] = None) -> StepRecord:
    """One forward step (``O.step``) that keeps its record."""
    spec = ds.spec
    p0 = ds.p.copy()
    gf = O.p2g(p0, spec.grid, mass_eps=spec.mass_eps)
    mask, vel = O.dirichlet_nodes(spec.grid, spec.dirichlet, dt)
    pr = O.make_problem(p0, spec.grid, gf, dt, spec.gravity, mask, vel)
    tol = spec.newton_tol if newton_tol is None else newton_tol
    u = O.newton(pr, tol, spec.newton_max, spec.ls_max)
    ds.p = O.g2p(p0, spec.grid, u, dt)
    return StepRecord(p0, pr, u)


@dataclass
class StateBar:
    """Adjoints of a particle state (same shapes as the state)."""
    x: np.ndarray
    v: np.ndarray
    B: np.ndarray
    F: np.ndarray

    @classmethod
    def zeros_like(cls, p: O.Particles) -> "StateBar":
        return cls(np.zeros_like(p.x), np.zeros_like(p.v), np.zeros_like(p.B), np.zeros_like(p.F))


def _lame_derivatives(E: np.ndarray, nu: np.ndarray):
    """d mu / dE and d lam / dE of ``O.lame``."""
    return 1.0 / (2.0 * (1.0 + nu)), nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def step_adjoint(rec: StepRecord, out: StateBar):
    """Given the adjoint of s^{n+1}, returns (adjoint of s^n, dJ/dE of this
    step's solve)."""
    pr, p, u = rec.pr, rec.p, rec.u
    st, grid, dt = pr.st, pr.grid, pr.dt
    n, d = p.x.shape
    nn = grid.n_nodes
    Hs = stencil_hessian(p.x, grid, st)
    uk = u[st.node]                                      # (n, K, d)
    dxi = st.xi - p.x[:, None, :]                        # x_i - x_p
    # ---- G2P (x', v', B', F')
    xb, vb, Bb, Fb = out.x, out.v, out.B, out.F
    contrib = (st.N[:, :, None] * (xb + vb / dt)[:, None, :]
               + st.N[:, :, None] / dt * np.einsum("pab,pkb->pka", Bb, dxi)
               + np.einsum("pab,pcb,pkc->pka", Fb, p.F, st.dN))
    ubar = np.zeros((nn, d))
    for a in range(d):
        np.add.at(ubar[:, a], st.node, contrib[:, :, a])
    s_k = (np.einsum("pa,pka->pk", xb + vb / dt, uk)
           + np.einsum("pka,pab,pkb->pk", uk, Bb, dxi) / dt)
    x_bar = (xb + np.einsum("pka,pk->pa", st.dN, s_k)
             - np.einsum("pk,pba,pkb->pa", st.N, Bb, uk) / dt
             + np.einsum("pkab,pbc,pdc,pkd->pa", Hs, p.F, Fb, uk))
    A = np.eye(d)[None] + np.einsum("pka,pkb->pab", uk, st.dN)
    F_bar = np.einsum("pba,pbc->pac", A, Fb)
    # ---- the solve: K lam = u_bar on the free DOFs
    free = pr.free.reshape(-1)
    idx = np.nonzero(free)[0]
    lam = np.zeros(nn * d)
    if idx.size:
        Hm = O.hessian(pr, u)[idx][:, idx].tocsc()
        lam[idx] = spla.spsolve(Hm, ubar.reshape(-1)[idx])
    lam = lam.reshape(nn, d)
    lk = lam[st.node]
    Fh = O.deformation(p, st, u)
    P = O.pk1(Fh, pr.mu, pr.lam)
    Aq = O.dpdf(Fh, pr.mu, pr.lam)                       # [p, a, c, b, e] = dP_ac / dF_be
    Gl = np.einsum("pka,pkb->pab", lk, st.dN)
    X = np.einsum("pab,pbc->pac", Gl, p.F)
    Y = np.einsum("pacbe,pbe->pac", Aq, X)
    V = p.vol0
    F_bar -= V[:, None, None] * (np.einsum("pba,pbc->pac", A, Y) + np.einsum("pba,pbc->pac", Gl, P))
    FiT = np.linalg.inv(Fh).transpose(0, 2, 1)
    lnJ = np.log(np.linalg.det(Fh))
    mu_bar = -V * np.einsum("pab,pab->p", Fh - FiT, X)
    lam_bar = -V * lnJ * np.einsum("pab,pab->p", FiT, X)
    dmu, dlam = _lame_derivatives(p.E, p.nu)
    E_bar = mu_bar * dmu + lam_bar * dlam
    # Y^T u_k + P^T lam_k, pulled back through F and the stencil Hessian
    Z = np.einsum("pba,pkb->pka", Y, uk) + np.einsum("pba,pkb->pka", P, lk)
    x_bar -= V[:, None] * np.einsum("pkab,pbc,pkc->pa", Hs, p.F, Z)
    gf = pr.gf
    act = gf.active
    g_ext = (pr.fext[act] / gf.m[act, None])
    v_node_bar = np.zeros((nn, d))
    m_node_bar = np.zeros(nn)
    v_node_bar[act] = gf.m[act, None] / dt * lam[act]
    m_node_bar[act] = -np.sum(lam[act] * ((u[act] - dt * gf.vn[act]) / dt ** 2 - g_ext), axis=1)
    # ---- P2G: v_i = q_i / m_i
    q_bar = np.zeros((nn, d))
    q_bar[act] = v_node_bar[act] / gf.m[act, None]
    m_node_bar[act] -= np.sum(v_node_bar[act] * gf.vn[act], axis=1) / gf.m[act]
    qk = q_bar[st.node]
    mk = m_node_bar[st.node]
    mp = p.mass
    Dinv = 4.0 / grid.dx ** 2
    C = Dinv * p.B
    v_bar = mp[:, None] * np.einsum("pk,pka->pa", st.N, qk)
    B_bar = Dinv * mp[:, None, None] * np.einsum("pk,pka,pkb->pab", st.N, qk, dxi)
    vel_k = p.v[:, None, :] + np.einsum("pab,pkb->pka", C, dxi)
    x_bar += mp[:, None] * (np.einsum("pka,pk->pa", st.dN, np.einsum("pka,pka->pk", qk, vel_k) + mk)
                            - np.einsum("pk,pba,pkb->pa", st.N, C, qk))
    return StateBar(x_bar, v_bar, B_bar, F_bar), E_bar


def trajectory_gradient(spec, dt: float, n_steps: int, dJ_dx: np.ndarray,
                        newton_tol: Optional[float] = None):
    """Runs n_steps from spec's particles and returns (final particles,
    dJ/dE, adjoint of the initial state) for J with dJ/dx_final = dJ_dx."""
    ds = O.DomainState.create(spec)
    recs: List[StepRecord] = [record_step(ds, dt, newton_tol) for _ in range(n_steps)]
    bar = StateBar.zeros_like(ds.p)
    bar.x = np.array(dJ_dx, dtype=np.float64, copy=True)
    E_bar = np.zeros(ds.p.x.shape[0])
    for rec in reversed(recs):
        bar, eb = step_adjoint(rec, bar)
        E_bar += eb
    return ds.p, E_bar, bar
