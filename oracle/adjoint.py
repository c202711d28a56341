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


def g2p_adjoint(p: O.Particles, pr: O.Problem, u: np.ndarray, out: StateBar):
    """Transposed G2P, F update and advection (Eqs. g2p_v, g2p_B, F_update,
    advection) of particles p moved by grid displacement u: returns (u_bar on
    the grid, the direct x_bar and F_bar of p)."""
    st, grid, dt = pr.st, pr.grid, pr.dt
    n, d = p.x.shape
    Hs = stencil_hessian(p.x, grid, st)
    uk = u[st.node]
    dxi = st.xi - p.x[:, None, :]
    xb, vb, Bb, Fb = out.x, out.v, out.B, out.F
    contrib = (st.N[:, :, None] * (xb + vb / dt)[:, None, :]
               + st.N[:, :, None] / dt * np.einsum("pab,pkb->pka", Bb, dxi)
               + np.einsum("pab,pcb,pkc->pka", Fb, p.F, st.dN))
    ubar = np.zeros((grid.n_nodes, d))
    for a in range(d):
        np.add.at(ubar[:, a], st.node, contrib[:, :, a])
    s_k = (np.einsum("pa,pka->pk", xb + vb / dt, uk)
           + np.einsum("pka,pab,pkb->pk", uk, Bb, dxi) / dt)
    x_bar = (xb + np.einsum("pka,pk->pa", st.dN, s_k)
             - np.einsum("pk,pba,pkb->pa", st.N, Bb, uk) / dt
             + np.einsum("pkab,pbc,pdc,pkd->pa", Hs, p.F, Fb, uk))
    A = np.eye(d)[None] + np.einsum("pka,pkb->pab", uk, st.dN)
    F_bar = np.einsum("pba,pbc->pac", A, Fb)
    return ubar, x_bar, F_bar


@dataclass
class SolveBar:
    lam: np.ndarray        # (nn, d) adjoint solution, 0 off the free DOFs
    F: np.ndarray          # F_bar of the particles
    x: np.ndarray          # x_bar of the particles
    E: np.ndarray          # dJ/dE of the particles
    v_node: np.ndarray     # (nn, d) adjoint of the P2G velocity v_i
    m_node: np.ndarray     # (nn,) adjoint of the P2G mass m_i
    u_fixed: np.ndarray    # (nn, d) adjoint of the prescribed displacement on fixed DOFs


def solve_adjoint(pr: O.Problem, u: np.ndarray, ubar: np.ndarray) -> SolveBar:
    """Implicit function theorem at the converged solve g(u) = 0 of problem
    pr: K lam = u_bar on the free DOFs, then -lam . dg/dz for the particle
    inputs (F, mu, lam -> E, x), the nodal mass and velocity; and, for the
    prescribed displacement u_D of each fixed DOF, dJ/du_D = u_bar_D -
    (K lam)_D."""
    p, st, grid, dt = pr.p, pr.st, pr.grid, pr.dt
    n, d = p.x.shape
    nn = grid.n_nodes
    Hs = stencil_hessian(p.x, grid, st)
    uk = u[st.node]
    free = pr.free.reshape(-1)
    idx = np.nonzero(free)[0]
    lam = np.zeros(nn * d)
    Hfull = O.hessian(pr, u)
    if idx.size:
        lam[idx] = spla.spsolve(Hfull[idx][:, idx].tocsc(), ubar.reshape(-1)[idx])
    Klam = (Hfull @ lam).reshape(nn, d)
    lam = lam.reshape(nn, d)
    u_fixed_bar = np.where(pr.fixed, ubar - Klam, 0.0)
    lk = lam[st.node]
    Fh = O.deformation(p, st, u)
    P = O.pk1(Fh, pr.mu, pr.lam)
    Aq = O.dpdf(Fh, pr.mu, pr.lam)
    A = np.eye(d)[None] + np.einsum("pka,pkb->pab", uk, st.dN)
    Gl = np.einsum("pka,pkb->pab", lk, st.dN)
    X = np.einsum("pab,pbc->pac", Gl, p.F)
    Y = np.einsum("pacbe,pbe->pac", Aq, X)
    V = p.vol0
    F_bar = -V[:, None, None] * (np.einsum("pba,pbc->pac", A, Y) + np.einsum("pba,pbc->pac", Gl, P))
    FiT = np.linalg.inv(Fh).transpose(0, 2, 1)
    lnJ = np.log(np.linalg.det(Fh))
    mu_bar = -V * np.einsum("pab,pab->p", Fh - FiT, X)
    lam_bar = -V * lnJ * np.einsum("pab,pab->p", FiT, X)
    dmu, dlam = _lame_derivatives(p.E, p.nu)
    E_bar = mu_bar * dmu + lam_bar * dlam
    Z = np.einsum("pba,pkb->pka", Y, uk) + np.einsum("pba,pkb->pka", P, lk)
    x_bar = -V[:, None] * np.einsum("pkab,pbc,pkc->pa", Hs, p.F, Z)
    gf = pr.gf
    act = gf.active
    g_ext = pr.fext[act] / gf.m[act, None]
    v_node = np.zeros((nn, d))
    m_node = np.zeros(nn)
    v_node[act] = gf.m[act, None] / dt * lam[act]
    m_node[act] = -np.sum(lam[act] * ((u[act] - dt * gf.vn[act]) / dt ** 2 - g_ext), axis=1)
    return SolveBar(lam, F_bar, x_bar, E_bar, v_node, m_node, u_fixed_bar)


def p2g_adjoint(p: O.Particles, grid, gf: O.GridFields, v_node: np.ndarray, m_node: np.ndarray):
    """Transposed APIC P2G (Eq. p2g_transfer) with v_i = q_i / m_i on the
    active nodes: from the adjoints of v_i and m_i to (v_bar, B_bar, x_bar)
    of the particles."""
    st = O.stencil(p.x, grid)
    nn, d = v_node.shape
    act = gf.active
    q_bar = np.zeros((nn, d))
    m_bar = np.zeros(nn)
    q_bar[act] = v_node[act] / gf.m[act, None]
    m_bar[act] = m_node[act] - np.sum(v_node[act] * gf.vn[act], axis=1) / gf.m[act]
    qk = q_bar[st.node]
    mk = m_bar[st.node]
    mp = p.mass
    dxi = st.xi - p.x[:, None, :]
    Dinv = 4.0 / grid.dx ** 2
    C = Dinv * p.B
    v_bar = mp[:, None] * np.einsum("pk,pka->pa", st.N, qk)
    B_bar = Dinv * mp[:, None, None] * np.einsum("pk,pka,pkb->pab", st.N, qk, dxi)
    vel_k = p.v[:, None, :] + np.einsum("pab,pkb->pka", C, dxi)
    x_bar = mp[:, None] * (np.einsum("pka,pk->pa", st.dN, np.einsum("pka,pka->pk", qk, vel_k) + mk)
                           - np.einsum("pk,pba,pkb->pa", st.N, C, qk))
    return v_bar, B_bar, x_bar


def step_adjoint(rec: StepRecord, out: StateBar, ubar_extra: Optional[np.ndarray] = None,
                 m_node_extra: Optional[np.ndarray] = None):
    """Given the adjoint of s^{n+1}, returns (adjoint of s^n, dJ/dE of this
    step's solve, the SolveBar).  ``ubar_extra`` and ``m_node_extra`` add
    adjoints of the solved displacement and of the P2G mass that reach them
    by other routes (the coupling operators)."""
    pr, p, u = rec.pr, rec.p, rec.u
    ubar, x_bar, F_bar = g2p_adjoint(p, pr, u, out)
    if ubar_extra is not None:
        ubar = ubar + ubar_extra
    sb = solve_adjoint(pr, u, ubar)
    m_node = sb.m_node if m_node_extra is None else sb.m_node + m_node_extra
    v_bar, B_bar, x_p2g = p2g_adjoint(p, pr.grid, pr.gf, sb.v_node, m_node)
    return StateBar(x_bar + sb.x + x_p2g, v_bar, B_bar, F_bar + sb.F), sb.E, sb


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
        bar, eb, _ = step_adjoint(rec, bar)
        E_bar += eb
    return ds.p, E_bar, bar


# ----------------------------------------------------------------------------
# The coupled step (Alg. 1), differentiated through the iterations it ran
# ----------------------------------------------------------------------------

@dataclass
class FineSub:
    p: O.Particles          # fine state entering the sub-step
    pr: O.Problem           # its solve (P2G grid, receivers as Dirichlet DOFs)
    u: np.ndarray           # converged displacement


@dataclass
class SchwarzIter:
    prB: O.Problem          # the coarse solve of this iteration
    uB: np.ndarray
    fine: List[FineSub]


@dataclass
class SchwarzRecord:
    B0: O.Particles
    S0: O.Particles
    gfB: O.GridFields       # coarse P2G at t_n (shared by every coarse solve)
    gfS0: O.GridFields      # fine P2G at t_n (the k = 0 projection)
    sets: O.InterfaceSets
    iters: List[SchwarzIter]
    M: int
    dT: float
    eps_tol: float


def _problem(ds: O.DomainState, gf: O.GridFields, dt: float, extra_mask, extra_vel) -> O.Problem:
    """The Problem that ``O.solve_domain`` builds (physical rules win)."""
    spec = ds.spec
    mask, vel = O.dirichlet_nodes(spec.grid, spec.dirichlet, dt)
    add = extra_mask[:, None] & ~mask
    vel = np.where(add, extra_vel, vel)
    mask = mask | add
    return O.make_problem(ds.p, spec.grid, gf, dt, spec.gravity, mask, vel)


def record_schwarz_step(B: O.DomainState, S: O.DomainState, dT: float, sch,
                        newton_tol: Optional[float] = None,
                        n_iters: Optional[int] = None) -> SchwarzRecord:
    """``O.schwarz_step`` (step-average Pi) that keeps what its adjoint needs.
    With ``n_iters`` it runs exactly that many Schwarz iterations instead of
    stopping at convergence (to unroll the same iterations as another run)."""
    if sch.pi_source != 0:
        raise NotImplementedError("the adjoint follows the step-average projection")
    M = sch.M
    dt = dT / M
    gB, gS = B.spec.grid, S.spec.grid
    tolB = B.spec.newton_tol if newton_tol is None else newton_tol
    tolS = S.spec.newton_tol if newton_tol is None else newton_tol
    B0, snap = B.p.copy(), S.p.copy()
    gfB = O.p2g(B.p, gB, boundary_mass=True, mass_eps=B.spec.mass_eps)
    gfS = O.p2g(S.p, gS, boundary_mass=True, mass_eps=S.spec.mass_eps)
    sets = O.interface_sets(B, S, gfB, gfS, sch, dT)
    vGB = O.project_S2B(gB, gS, gfS, sets.recvB, sch.eps_tol)
    vGS = O.interp_B2S(gB, gS, gfB.vn, sets.recvS)
    vSn = vGS.copy()
    iters: List[SchwarzIter] = []
    for k in range(sch.k_max + 1 if n_iters is None else n_iters):
        prB = _problem(B, gfB, dT, sets.recvB, vGB)
        uB = O.newton(prB, tolB, B.spec.newton_max, B.spec.ls_max)
        vB_new = np.where(gfB.active[:, None], uB / dT, 0.0)
        S.p = snap.copy()
        gf = O.p2g(S.p, gS, mass_eps=S.spec.mass_eps)
        vSnp1 = O.interp_B2S(gB, gS, vB_new, sets.recvS)
        fine, solved, vels = [], [], []
        for m in range(1, M + 1):
            bc = O.time_interp(vSn, vSnp1, m, M)
            pr = _problem(S, gf, dt, sets.recvS, bc)
            uS = O.newton(pr, tolS, S.spec.newton_max, S.spec.ls_max)
            fine.append(FineSub(S.p.copy(), pr, uS))
            solved.append(gf)
            vels.append(uS / dt)
            S.p = O.g2p(S.p, gS, uS, dt)
            gf = O.p2g(S.p, gS, mass_eps=S.spec.mass_eps)
        iters.append(SchwarzIter(prB, uB, fine))
        vGB_new = O.project_S2B(gB, gS, O.substep_average(solved, vels), sets.recvB, sch.eps_tol)
        rB = O.rel_change(vGB_new, vGB, sets.recvB)
        rS = O.rel_change(vSnp1, vGS, sets.recvS)
        vGB, vGS = vGB_new, vSnp1
        if n_iters is None and k >= 1 and rB <= sch.eps_conv and rS <= sch.eps_conv:
            break
    B.p = O.g2p(B.p, gB, uB, dT)
    return SchwarzRecord(B0, snap, gfB, gfS, sets, iters, M, dT, sch.eps_tol)


def _coupling_weights(gB, gS):
    """For every fine node j: its coarse support nodes (nS, K) and the
    weights N_I(x_Sj), zero where the support leaves the coarse box."""
    xS = O.node_positions(gS)
    st = O.stencil(xS, gB, check=False)
    res = np.asarray(gB.res)
    ok = np.all((st.nodes3 >= 0) & (st.nodes3 < res[None, None]), axis=2)
    return np.where(ok, st.node, 0), st.N * ok


def interp_adjoint(gB, gS, v_bar: np.ndarray, recvS: np.ndarray) -> np.ndarray:
    """Transposed I_{B->S} (Eq. interp_BtoS) over the fine receivers."""
    node, w = _coupling_weights(gB, gS)
    out = np.zeros((gB.n_nodes, v_bar.shape[1]))
    idx = np.nonzero(recvS)[0]
    for a in range(v_bar.shape[1]):
        np.add.at(out[:, a], node[idx], w[idx] * v_bar[idx, a][:, None])
    return out


def proj_adjoint(gB, gS, m: np.ndarray, vn: np.ndarray, active: np.ndarray, recvB: np.ndarray,
                 eps_tol: float, v_bar: np.ndarray):
    """Transposed Pi_{S->B} (Eq. spatial_projection) on the coarse receivers,
    Pi_I = sum_j N_Ij (m v)_j / (sum_j N_Ij m_j + eps_tol): returns the
    adjoints of the fine nodal momentum (m v)_j and mass m_j."""
    num, den = O.projection_sums(gB, gS, m, vn, active)
    dd = den + eps_tol
    num_bar = np.where(recvB[:, None], v_bar / dd[:, None], 0.0)
    den_bar = np.where(recvB, -np.sum(v_bar * num, axis=1) / dd ** 2, 0.0)
    node, w = _coupling_weights(gB, gS)
    mv_bar = np.einsum("jk,jka->ja", w, num_bar[node])
    m_bar = np.einsum("jk,jk->j", w, den_bar[node])
    mv_bar[~active] = 0.0
    m_bar[~active] = 0.0
    return mv_bar, m_bar


def schwarz_adjoint(rec: SchwarzRecord, barB: StateBar, barS: StateBar):
    """Reverse of one recorded coupled step: from the adjoints of the coarse
    and fine states after it to those before it and to dJ/dE of both
    particle sets.  The iterations are unrolled as they ran (their number and
    the receiver sets held fixed)."""
    gB, gS = rec.iters[0].prB.grid, rec.iters[0].fine[0].pr.grid
    M, dT = rec.M, rec.dT
    dt = dT / M
    d = rec.B0.x.shape[1]
    recvB, recvS = rec.sets.recvB, rec.sets.recvS
    K = len(rec.iters) - 1
    B0bar = StateBar.zeros_like(rec.B0)
    S0bar = StateBar.zeros_like(rec.S0)
    EB = np.zeros(rec.B0.x.shape[0])
    ES = np.zeros(rec.S0.x.shape[0])
    vBn_bar = np.zeros((gB.n_nodes, d))      # coarse P2G velocity at t_n
    mBn_bar = np.zeros(gB.n_nodes)          # coarse P2G mass at t_n
    vSn_bar = np.zeros((gS.n_nodes, d))      # I(v_B^n) on the fine receivers
    # post-convergence coarse G2P with the last coarse solution
    last = rec.iters[K]
    ubarB, xb, Fb = g2p_adjoint(rec.B0, last.prB, last.uB, barB)
    B0bar.x += xb
    B0bar.F += Fb
    inject = [None] * (K + 1)   # Pi adjoints reaching fine iteration k
    for k in range(K, -1, -1):
        it = rec.iters[k]
        bar = barS if k == K else StateBar.zeros_like(rec.S0)
        vSnp1_bar = np.zeros((gS.n_nodes, d))
        for m in range(M - 1, -1, -1):
            sub = it.fine[m]
            u_extra = m_extra = None
            if inject[k] is not None:
                mvb, mdb = inject[k]
                gf = sub.pr.gf
                act = gf.active
                u_extra = np.where(act[:, None], gf.m[:, None] / (M * dt) * mvb, 0.0)
                m_extra = np.where(act, (np.sum(sub.u / dt * mvb, axis=1) + mdb) / M, 0.0)
            bar, eb, sb = step_adjoint(StepRecord(sub.p, sub.pr, sub.u), bar, u_extra, m_extra)
            ES += eb
            a = (m + 1) / M
            uDb = np.where(recvS[:, None], sb.u_fixed, 0.0)
            vSn_bar += (1.0 - a) * dt * uDb
            vSnp1_bar += a * dt * uDb
        S0bar = StateBar(S0bar.x + bar.x, S0bar.v + bar.v, S0bar.B + bar.B, S0bar.F + bar.F)
        # v_S^{n+1} = I(v_B^(k+1)), v_B^(k+1) = u_B^(k) / dT on the active coarse nodes
        vB_bar = interp_adjoint(gB, gS, vSnp1_bar, recvS)
        ub = np.where(rec.gfB.active[:, None], vB_bar / dT, 0.0)
        if k == K:
            ub = ub + ubarB
        sbB = solve_adjoint(it.prB, it.uB, ub)
        EB += sbB.E
        B0bar.x += sbB.x
        B0bar.F += sbB.F
        vBn_bar += sbB.v_node
        mBn_bar += sbB.m_node
        vGB_bar = np.where(recvB[:, None], dT * sbB.u_fixed, 0.0)
        if k >= 1:
            # v_GammaB^(k) = Pi of fine iteration k-1's step average
            prev = rec.iters[k - 1]
            grids = [f.pr.gf for f in prev.fine]
            vels = [f.u / dt for f in prev.fine]
            src = O.substep_average(grids, vels)
            inject[k - 1] = proj_adjoint(gB, gS, src.m, src.vn, src.active, recvB, rec.eps_tol, vGB_bar)
        else:
            # v_GammaB^(0) = Pi of the fine P2G at t_n
            g0 = rec.gfS0
            mvb, mdb = proj_adjoint(gB, gS, g0.m, g0.vn, g0.active, recvB, rec.eps_tol, vGB_bar)
            v_node = g0.m[:, None] * mvb
            m_node = np.sum(g0.vn * mvb, axis=1) + mdb
            vb, Bb, xb = p2g_adjoint(rec.S0, gS, g0, v_node, m_node)
            S0bar = StateBar(S0bar.x + xb, S0bar.v + vb, S0bar.B + Bb, S0bar.F)
    # v_S^n = I(v_B^n), and the coarse P2G at t_n
    vBn_bar += interp_adjoint(gB, gS, vSn_bar, recvS)
    vb, Bb, xb = p2g_adjoint(rec.B0, gB, rec.gfB, vBn_bar, mBn_bar)
    B0bar = StateBar(B0bar.x + xb, B0bar.v + vb, B0bar.B + Bb, B0bar.F)
    return B0bar, S0bar, EB, ES
