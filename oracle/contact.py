"""Unilateral frictionless contact of a body with a rigid plane, for the
oracle (test infrastructure: only the tests, the smoke check and the
bench's CPU baseline import ``oracle``).

Reading of the rigid plane of Sec. 4.2 (the paper does not spell out its
contact treatment): the plane acts on the normal (y) component of the grid
nodes at or below it.  Over one implicit step the grid displacement u
minimises E_h subject to u_iy >= 0 on those nodes (a node may leave the
plane, not enter it), and the tangential components stay free
(frictionless).  The constrained minimum satisfies the Signorini
conditions with the multiplier lambda_i = dE_h/du_iy (the plane's force on
node i): lambda_i >= 0, u_iy >= 0 and lambda_i u_iy = 0.  It is found by a
primal-dual active set: solve with u_iy = 0 held on the active nodes,
release the active nodes whose multiplier is negative (the plane would
have to pull) and activate the free nodes that moved into the plane;
repeat until the set no longer changes.
"""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np

from . import osmpm_oracle as O


def plane_gaps(p: O.Particles, grid: O.Grid, plane_nodes: np.ndarray, spacing: float,
               y0: float = 0.0) -> np.ndarray:
    """Per candidate node, the distance from the plane y = y0 up to the
    body's lower surface over the node: the lowest particle whose x lies
    within one particle spacing of the node's x, minus half a spacing
    (clamped at 0; +inf where no particle lies over the node)."""
    xn = O.node_positions(grid)
    gap = np.full(len(xn), np.inf)
    for i in np.nonzero(plane_nodes)[0]:
        col = np.abs(p.x[:, 0] - xn[i, 0]) <= spacing
        if col.any():
            gap[i] = max(0.0, p.x[col, 1].min() - 0.5 * spacing - y0)
    return gap


def solve_with_plane(ds: O.DomainState, gf: O.GridFields, dt: float, plane_nodes: np.ndarray,
                     gap: np.ndarray, max_sets: int = 50,
                     stats: Optional[O.NewtonStats] = None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """One implicit solve of ``ds`` with the unilateral plane on the
    candidate nodes ``plane_nodes`` ((n_nodes,) bool): u_iy >= -gap_i.
    Returns (u, active set, multiplier lambda per node (0 off the active
    set))."""
    spec = ds.spec
    mask, vel = O.dirichlet_nodes(spec.grid, spec.dirichlet, dt)
    cand = plane_nodes & gf.active & ~mask[:, 1] & np.isfinite(gap)
    act = cand & (gap <= 0.0)              # start from the closed gaps
    for _ in range(max_sets):
        m = mask.copy()
        v = vel.copy()
        m[act, 1] = True
        v[act, 1] = -gap[act] / dt
        pr = O.make_problem(ds.p, spec.grid, gf, dt, spec.gravity, m, v)
        u = O.newton(pr, spec.newton_tol, spec.newton_max, spec.ls_max, stats)
        lam = np.where(act, O.gradient(pr, u)[:, 1], 0.0)
        release = act & (lam < 0.0)
        enter = cand & ~act & (u[:, 1] < -gap)
        if not release.any() and not enter.any():
            return u, act, lam
        act = (act & ~release) | enter
    raise O.OracleError("the contact active set did not settle")


def step_with_plane(ds: O.DomainState, dt: float, plane_nodes: np.ndarray, spacing: float,
                    stats: Optional[O.NewtonStats] = None) -> Tuple[np.ndarray, np.ndarray]:
    """One backward-Euler MPM step with the unilateral plane: P2G, the
    constrained solve, G2P.  Returns (active set, multiplier per node)."""
    gf = O.p2g(ds.p, ds.spec.grid, mass_eps=ds.spec.mass_eps)
    gap = plane_gaps(ds.p, ds.spec.grid, plane_nodes, spacing)
    u, act, lam = solve_with_plane(ds, gf, dt, plane_nodes, gap, stats=stats)
    ds.p = O.g2p(ds.p, ds.spec.grid, u, dt)
    return act, lam


def settle_hertz(dx: float, ppc_1d: int, indent: float, n_steps: int = 10, dt: float = 0.02,
                 dt_settle: float = 0.2, max_settle: int = 200):
    """The cylinder of Sec. 4.2 (``workloads.hertz_rigid_single``) pressed
    onto the rigid plane y = 0 by its flat face (``indent`` over ``n_steps``
    steps of dt, the pushed node rows following the face down), then held
    and settled with steps of dt_settle.  Every step is kinetically damped
    (v and B zeroed after it) and solves the unilateral contact
    (``step_with_plane``) with the plane candidates of the workload and the
    particle spacing dx/ppc_1d; settling stops at the first step after which
    the largest particle speed is below 1e-6.  Returns (spec, plane nodes,
    grid fields, gaps, active set, multipliers, last u, settled state,
    settle steps)."""
    import dataclasses
    from paper_2605_09097_gb300 import workloads as W
    spec, plane = W.hertz_rigid_single(dx=dx, ppc_1d=ppc_1d, indent=indent, n_steps=n_steps, dt=dt)
    ds = O.DomainState.create(spec)
    h = dx / ppc_1d
    push = spec.dirichlet[0]
    for k in range(n_steps):
        lo = (push.lo[0], push.lo[1] - k * indent / n_steps)
        ds.spec = dataclasses.replace(spec, dirichlet=[dataclasses.replace(push, lo=lo)])
        step_with_plane(ds, dt, plane, h)
        ds.p.v[:] = 0.0
        ds.p.B[:] = 0.0
    lo = (push.lo[0], push.lo[1] - indent)
    ds.spec = dataclasses.replace(spec, dirichlet=[dataclasses.replace(push, lo=lo, vel=(0.0, 0.0, 0.0))])
    for k in range(max_settle):
        gf = O.p2g(ds.p, spec.grid, mass_eps=spec.mass_eps)
        gap = plane_gaps(ds.p, spec.grid, plane, h)
        u, act, lam = solve_with_plane(ds, gf, dt_settle, plane, gap)
        ds.p = O.g2p(ds.p, spec.grid, u, dt_settle)
        vmax = np.abs(ds.p.v).max()
        ds.p.v[:] = 0.0
        ds.p.B[:] = 0.0
        if vmax < 1e-6:
            return spec, plane, gf, gap, act, lam, u, ds, k + 1
    raise O.OracleError("the contact did not settle")
