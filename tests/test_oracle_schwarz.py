"""Pins of the oracle's Schwarz operators and loop (Sec. 3, Alg. 1) against
facts the paper and the mathematics fix (no GPU)."""
import dataclasses

import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W


def _inclusion_small():
    return W.inclusion(dx_S=0.02, M=2)


def test_projection_of_constant_field_is_constant():
    cB, cS, sch, dT = _inclusion_small()
    gfS = O.p2g(cS.particles, cS.grid)
    c = np.array([0.3, -0.7])
    gfS.vn = np.where(gfS.active[:, None], c[None], 0.0)
    num, den = O.projection_sums(cB.grid, cS.grid, gfS.m, gfS.vn, gfS.active)
    recv = den > sch.tau_B
    assert recv.sum() > 10
    v = O.project_S2B(cB.grid, cS.grid, gfS, recv, sch.eps_tol)
    np.testing.assert_allclose(v[recv], np.broadcast_to(c, v[recv].shape), rtol=1e-10)
    assert np.all(v[~recv] == 0)


def test_interpolation_reproduces_linear_field():
    cB, cS, _, _ = _inclusion_small()
    xB = O.node_positions(cB.grid)
    xS = O.node_positions(cS.grid)
    a = np.array([0.2, -0.1])
    C = np.array([[0.5, -1.5], [2.0, 0.25]])
    vB = a[None] + xB @ C.T
    recv = np.zeros(cS.grid.n_nodes, bool)
    recv[::7] = True
    v = O.interp_B2S(cB.grid, cS.grid, vB, recv)
    np.testing.assert_allclose(v[recv], a[None] + xS[recv] @ C.T, atol=1e-14)


def test_temporal_interpolation_is_exact_for_linear_data():
    v0, v1 = np.array([1.0, -2.0]), np.array([3.0, 6.0])
    for M in (1, 2, 4):
        for m in range(1, M + 1):
            t = m / M
            np.testing.assert_allclose(O.time_interp(v0, v1, m, M), v0 + t * (v1 - v0), atol=1e-15)
    np.testing.assert_array_equal(O.time_interp(v0, v1, 2, 2), v1)


@pytest.mark.parametrize("dxs,period", [(0.01, 5), (0.02, 5)])
def test_coincident_nodes_on_nested_and_nonnested_grids(dxs, period):
    cB, cS, _, _ = W.inclusion(dx_S=dxs)
    j = O.coincident_fine_node(cB.grid, cS.grid)
    xB = O.node_positions(cB.grid)
    inside = np.all((xB >= 0.3 - 1e-12) & (xB <= 0.7 + 1e-12), axis=1)
    # dx_B / dx_S = 5 (nested): every coarse node in the box coincides;
    # 2.5 (non-nested): only every second coarse node does
    if dxs == 0.01:
        assert np.all(j[inside] >= 0)
    else:
        ii = np.rint(xB[inside] / 0.05).astype(int)
        expect = np.all(ii % 2 == 0, axis=1)
        np.testing.assert_array_equal(j[inside] >= 0, expect)
    xS = O.node_positions(cS.grid)
    ok = j >= 0
    np.testing.assert_allclose(xS[j[ok]], xB[ok], atol=1e-12)
    assert np.all(~inside[~ok] | (j[~ok] < 0))


def test_rel_change_reading():
    mask = np.array([True, True, False])
    new = np.array([[3.0, 4.0], [0.0, 0.0], [9.0, 9.0]])
    old = np.zeros_like(new)
    assert O.rel_change(new, old, mask) == 1.0
    # zero denominator: absolute norm
    assert O.rel_change(np.zeros_like(new), new, mask) == 5.0
    # empty set: 0
    assert O.rel_change(new, old, np.zeros(3, bool)) == 0.0


def test_no_boundary_nodes_decouples_domains_exactly():
    """tau_Gamma = inf: no boundary node on either grid, so each domain takes
    its own standalone solve: P_B one step of dT, P_S M steps of dT/M."""
    cB, cS, sch, dT = _inclusion_small()
    sch = dataclasses.replace(sch, tau_B=np.inf, tau_S=np.inf, k_max=3)
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    st = O.SchwarzStats()
    O.schwarz_step(B, S, dT, sch, st)
    B1, S1 = O.DomainState.create(cB), O.DomainState.create(cS)
    O.step(B1, dT)
    for _ in range(sch.M):
        O.step(S1, dT / sch.M)
    np.testing.assert_array_equal(B.p.x, B1.p.x)
    np.testing.assert_array_equal(S.p.x, S1.p.x)
    np.testing.assert_array_equal(S.p.F, S1.p.F)
    assert st.iters == 2 and st.converged


def test_identical_domains_reduce_to_single_domain():
    """Identical grid and particles, M = 1: every boundary node coincides with
    one of the other grid and the mass tie makes B the donor (Eq.
    overlap_donor), so Gamma_hat_B is empty, the coarse result equals the
    single-domain step exactly and the loop stops at k = 1."""
    spec = W.perturb(W.block(2, n_cells=(6, 4), dx=0.1, E=1e5, gravity=(0.0, -9.81)), 4)
    Bs, Ss, sch = W.identical_pair(spec, M=1)
    B, S = O.DomainState.create(Bs), O.DomainState.create(Ss)
    st = O.SchwarzStats()
    so = {}
    O.schwarz_step(B, S, 0.01, sch, st, so)
    assert so["sets"].recvB.sum() == 0
    assert so["sets"].recvS.sum() > 0
    ref = O.DomainState.create(spec)
    O.step(ref, 0.01)
    np.testing.assert_array_equal(B.p.x, ref.p.x)
    np.testing.assert_array_equal(B.p.F, ref.p.F)
    assert st.iters == 2 and st.converged
    # the fine copy is driven by I(v_B) on its receivers (a smoothing, not
    # an identity for the quadratic B-spline): close, not equal
    disp = np.abs(ref.p.x - spec.particles.x).max()
    dev = np.abs(S.p.x - ref.p.x).max()
    assert 0 < dev < disp


def test_schwarz_residuals_decay_geometrically():
    """Sec. 2.3: the alternating iteration contracts; on the small inclusion
    both interface residuals fall by a roughly constant factor < 1."""
    cB, cS, sch, dT = _inclusion_small()
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    st = O.SchwarzStats()
    O.schwarz_step(B, S, dT, sch, st)
    h = np.array(st.history)
    assert st.converged and st.iters < sch.k_max
    assert st.r_B <= sch.eps_conv and st.r_S <= sch.eps_conv
    ratios = h[4:, 0] / h[3:-1, 0]
    assert np.all(ratios < 0.9)


def test_substep_average_of_free_fall_is_mid_step_velocity():
    """Backward Euler on a stress-free block under gravity g gives the uniform
    grid velocity v^(m) = m g dt after sub-step m (E_h is minimised by the
    uniform u = dt v + dt^2 g, where F = I and the stress vanishes).  Over a
    coarse step of M = 2 sub-steps the fine motion is dT * 1.5 g dt, so the
    step-averaged velocity that feeds Pi is 1.5 g dt on every active node,
    not the 2 g dt of the last sub-step."""
    g = np.array([0.0, -9.81])
    spec = W.block(2, n_cells=(10, 8), dx=0.1, E=1e5, gravity=tuple(g))
    ds = O.DomainState.create(spec)
    dt, M = 0.01, 2
    grids, vels = [], []
    x0 = ds.p.x.copy()
    for m in range(1, M + 1):
        gf = O.p2g(ds.p, spec.grid, mass_eps=spec.mass_eps)
        u = O.solve_domain(ds, gf, dt)
        v = u / dt
        np.testing.assert_allclose(v[gf.active], np.broadcast_to(m * g * dt, v[gf.active].shape),
                                   atol=1e-9)
        grids.append(gf)
        vels.append(v)
        ds.p = O.g2p(ds.p, spec.grid, u, dt)
    avg = O.substep_average(grids, vels)
    m1 = np.where(grids[0].active, grids[0].m, 0.0)
    m2 = np.where(grids[1].active, grids[1].m, 0.0)
    # mass and momentum are the means over the two sub-steps
    np.testing.assert_allclose(avg.m, 0.5 * (m1 + m2), rtol=1e-14)
    np.testing.assert_allclose(avg.mv, 0.5 * (m1[:, None] * vels[0] + m2[:, None] * vels[1]),
                               rtol=1e-13, atol=1e-18)
    np.testing.assert_array_equal(avg.active, grids[0].active | grids[1].active)
    # interior nodes: two particles per cell along each axis make the nodal
    # mass invariant under the fall (partition of unity on each half-lattice),
    # so the average is exactly the mid-step velocity 1.5 g dt
    inner = grids[0].active & grids[1].active & (np.abs(m1 - m2) <= 1e-12 * np.maximum(m1, m2))
    assert inner.sum() >= 20
    np.testing.assert_allclose(avg.vn[inner], np.broadcast_to(1.5 * g * dt, avg.vn[inner].shape),
                               atol=1e-12)
    # edge nodes: a convex combination of g dt and 2 g dt
    vy = avg.vn[avg.active, 1]
    assert np.all(vy <= g[1] * dt + 1e-12) and np.all(vy >= 2 * g[1] * dt - 1e-12)
    # the particles moved by dT times the mid-step velocity
    np.testing.assert_allclose(ds.p.x - x0, np.broadcast_to(M * dt * 1.5 * g * dt, x0.shape), atol=1e-12)


def test_substep_average_with_one_substep_is_the_solved_grid():
    spec = W.perturb(W.block(2, n_cells=(5, 4), dx=0.1, E=1e5, gravity=(0.0, -9.81)), 7)
    ds = O.DomainState.create(spec)
    gf = O.p2g(ds.p, spec.grid, mass_eps=spec.mass_eps)
    u = O.solve_domain(ds, gf, 0.01)
    avg = O.substep_average([gf], [u / 0.01])
    np.testing.assert_array_equal(avg.active, gf.active)
    np.testing.assert_allclose(avg.vn[gf.active], (u / 0.01)[gf.active], rtol=1e-13, atol=1e-15)


def _brute_boundary_mass(p, grid):
    """Boundary-particle mass per node by a loop over particles and their
    3^d stencil nodes, B-spline weights from the 1D definition."""
    def w1(r):
        r = abs(r)
        return 0.75 - r * r if r < 0.5 else (0.5 * (1.5 - r) ** 2 if r < 1.5 else 0.0)
    d = grid.dim
    res = np.asarray(grid.res)
    bm = np.zeros(int(np.prod(res)))
    for q in np.nonzero(p.flags & 1)[0]:
        t = (p.x[q] - np.asarray(grid.origin[:d])) / grid.dx
        base = np.floor(t - 0.5).astype(int)
        for off in np.ndindex(*(3,) * d):
            node = base + np.array(off)
            w = np.prod([w1(t[a] - node[a]) for a in range(d)])
            flat = node[0] + res[0] * (node[1] + (res[1] * node[2] if d == 3 else 0))
            bm[flat] += p.mass[q] * w
    return bm


def test_interface_sets_follow_the_definitions():
    """Gamma (Eq. boundary_grid_set) holds the active nodes that carry more
    than tau of boundary-particle mass (checked against a brute-force
    boundary mass); after arbitration (Eq. overlap_donor) no coincident pair
    receives on both sides; receivers lie where the outer particle layers
    are (fine: around r = 0.15; coarse: around the hole r = 0.1, inside the
    fine region) and never on nodes with a physical Dirichlet rule."""
    cB, cS, sch, dT = _inclusion_small()
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    gfB = O.p2g(B.p, cB.grid, boundary_mass=True, mass_eps=cB.mass_eps)
    gfS = O.p2g(S.p, cS.grid, boundary_mass=True, mass_eps=cS.mass_eps)
    for gf, st, tau in ((gfB, B, sch.tau_B), (gfS, S, sch.tau_S)):
        bm = _brute_boundary_mass(st.p, st.spec.grid)
        np.testing.assert_allclose(gf.bm, bm, rtol=1e-12, atol=1e-15 * bm.max())
        assert np.array_equal(O.boundary_sets(gf, tau), gf.active & (bm > tau))
    sets = O.interface_sets(B, S, gfB, gfS, sch, dT)
    assert sets.recvB.any() and sets.recvS.any()
    assert not (sets.recvB & ~sets.gammaB).any() and not (sets.recvS & ~sets.gammaS).any()
    j = O.coincident_fine_node(cB.grid, cS.grid)
    pair = (j >= 0) & sets.recvB
    assert not sets.recvS[j[pair]].any()
    xS = O.node_positions(cS.grid)
    rS = np.hypot(xS[sets.recvS, 0] - 0.5, xS[sets.recvS, 1] - 0.5)
    reach = 1.5 * np.sqrt(2) * cS.grid.dx
    assert rS.min() >= 0.15 - cS.grid.dx / 2 - reach and rS.max() <= 0.15 + reach
    xB = O.node_positions(cB.grid)
    rB = np.hypot(xB[sets.recvB, 0] - 0.5, xB[sets.recvB, 1] - 0.5)
    assert rB.max() <= 0.125 + 1.5 * np.sqrt(2) * cB.grid.dx
    assert rB.max() <= 0.15 + 1.5 * np.sqrt(2) * cS.grid.dx   # fed by the fine projection
    mB, _ = O.dirichlet_nodes(cB.grid, cB.dirichlet, dT)
    assert not (sets.recvB & mB.any(axis=1)).any()


def test_particles_advance_once_per_global_step():
    """Sec. 3.5: after convergence the fine particles keep the state of the
    last iteration's sub-steps (they are not reset to the snapshot), and the
    coarse particles take one G2P with the last coarse solve.  Under the top
    edge's 1e-3 downward displacement per step, the fine particles have
    moved downward (a reset would leave them at rest), and no coarse particle
    moves by more than the prescribed 1e-3 (a G2P per Schwarz iteration
    would move the top rows by about k times as much)."""
    cB, cS, sch, dT = _inclusion_small()
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    st = O.SchwarzStats()
    O.schwarz_step(B, S, dT, sch, st)
    assert st.converged and st.iters >= 2
    dS = S.p.x - cS.particles.x
    dB = B.p.x - cB.particles.x
    upper = cS.particles.x[:, 1] > 0.55
    assert dS[upper, 1].mean() < -1e-6
    assert np.abs(dB).max() <= 1e-3 * (1 + 1e-9)
    top = cB.particles.x[:, 1] > 0.85
    assert dB[top, 1].mean() < -0.5e-3


def _brute_coarse_support_active(gB, gS, activeB):
    """Per fine node, by loops: its position o_S + j dx_S from the integer
    multi-index, the coarse base node floor((x - o_B)/dx_B - 1/2) per axis,
    and all 3^d coarse nodes base + {0, 1, 2}^d inside the coarse box and
    active."""
    d = gS.dim
    resB = [int(r) for r in gB.res[:d]]
    out = np.zeros(int(np.prod(gS.res)), dtype=bool)
    for flat, j in enumerate(np.ndindex(*reversed([int(r) for r in gS.res[:d]]))):
        j = j[::-1]  # x fastest
        x = [gS.origin[a] + j[a] * gS.dx for a in range(d)]
        base = [int(np.floor((x[a] - gB.origin[a]) / gB.dx - 0.5)) for a in range(d)]
        ok = True
        for off in np.ndindex(*(3,) * d):
            node = [base[a] + off[a] for a in range(d)]
            if any(node[a] < 0 or node[a] >= resB[a] for a in range(d)):
                ok = False
                break
            I = node[0] + resB[0] * (node[1] + (resB[1] * node[2] if d == 3 else 0))
            if not activeB[I]:
                ok = False
                break
        out[flat] = ok
    return out


def test_coarse_support_filter_matches_brute_force():
    """The Gamma_hat_S filter (coarse support of a fine node inside the box
    and active) against the brute-force loop, on the inclusion's coarse
    active set and on seeded random active sets over a fine grid that
    reaches past the coarse box.  The random sets include fine nodes whose
    only inactive support node lies in the third stencil row of an axis, so
    a filter that dropped that row (or tested "inside" without "active", or
    the reverse) would fail."""
    cB, cS, _, _ = _inclusion_small()
    gB, gS = cB.grid, cS.grid
    gfB = O.p2g(cB.particles, gB, mass_eps=cB.mass_eps)
    got = O.coarse_support_active(gB, gS, gfB.active)
    want = _brute_coarse_support_active(gB, gS, gfB.active)
    assert got.any() and (~got).any()
    np.testing.assert_array_equal(got, want)
    # a fine grid hanging over the coarse box (origin below it, reaching past it)
    gS2 = W.Grid(2, (gB.origin[0] - 3.3 * gS.dx, gB.origin[1] + 0.37 * gB.dx), gS.dx,
                 (int(round(1.2 / gS.dx)), int(round(0.6 / gS.dx))))
    rng = np.random.default_rng(7)
    third_row_hits = 0
    for p_active in (0.97, 0.9):
        act = rng.random(gB.n_nodes) < p_active
        got = O.coarse_support_active(gB, gS2, act)
        want = _brute_coarse_support_active(gB, gS2, act)
        np.testing.assert_array_equal(got, want)
        # fine nodes that only the third row of some axis rules out
        xs = O.node_positions(gS2)
        t = (xs - np.asarray(gB.origin)[None]) / gB.dx
        base = np.floor(t - 0.5).astype(int)
        inside = np.all((base >= 0) & (base + 2 < np.asarray(gB.res)[None]), axis=1)
        for k in np.nonzero(inside & ~got)[0][:400]:
            two = True
            for off in np.ndindex(2, 2):
                I = (base[k, 0] + off[0]) + gB.res[0] * (base[k, 1] + off[1])
                two &= bool(act[I])
            third_row_hits += two
    assert third_row_hits > 0
