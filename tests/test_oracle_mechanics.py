"""Pins of the oracle's constitutive law, incremental potential, Newton
solver and single-domain step against textbook facts (no GPU)."""
import dataclasses

import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W


def _rand_F(n, d, scale, seed):
    rng = np.random.default_rng(seed)
    return np.eye(d)[None] + scale * rng.standard_normal((n, d, d))


def test_lame_inverse_relations():
    E = np.array([1e6, 2e5, 3.3e7])
    nu = np.array([0.3, 0.4, 0.1])
    mu, lam = O.lame(E, nu)
    np.testing.assert_allclose(mu * (3 * lam + 2 * mu) / (lam + mu), E, rtol=1e-14)
    np.testing.assert_allclose(lam / (2 * (lam + mu)), nu, rtol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_rest_state_is_stress_free(d):
    F = np.broadcast_to(np.eye(d), (3, d, d)).copy()
    mu, lam = np.full(3, 2.0), np.full(3, 3.0)
    np.testing.assert_array_equal(O.psi(F, mu, lam), 0.0)
    np.testing.assert_allclose(O.pk1(F, mu, lam), 0.0, atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("scale", [0.05, 0.3])
def test_pk1_is_derivative_of_psi(d, scale):
    F = _rand_F(6, d, scale, 11 + d)
    mu, lam = np.full(6, 1.3), np.full(6, 2.1)
    P = O.pk1(F, mu, lam)
    h = 1e-6
    for a in range(d):
        for b in range(d):
            E = np.zeros((d, d))
            E[a, b] = h
            fd = (O.psi(F + E, mu, lam) - O.psi(F - E, mu, lam)) / (2 * h)
            np.testing.assert_allclose(P[:, a, b], fd, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("d", [2, 3])
def test_tangent_is_derivative_of_pk1(d):
    F = _rand_F(5, d, 0.2, 21 + d)
    mu, lam = np.full(5, 1.3), np.full(5, 2.1)
    A = O.dpdf(F, mu, lam)
    h = 1e-6
    for b in range(d):
        for e in range(d):
            E = np.zeros((d, d))
            E[b, e] = h
            fd = (O.pk1(F + E, mu, lam) - O.pk1(F - E, mu, lam)) / (2 * h)
            np.testing.assert_allclose(A[:, :, :, b, e], fd, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("d", [2, 3])
def test_small_strain_limit_is_hooke(d):
    rng = np.random.default_rng(3)
    S = rng.standard_normal((4, d, d))
    S = 0.5 * (S + np.transpose(S, (0, 2, 1)))
    eps = 1e-5
    mu, lam = np.full(4, 1.7), np.full(4, 0.9)
    e = eps * S
    hooke = 0.5 * lam * np.trace(e, axis1=1, axis2=2) ** 2 + mu * np.sum(e * e, axis=(1, 2))
    got = O.psi(np.eye(d)[None] + e, mu, lam)
    np.testing.assert_allclose(got, hooke, rtol=1e-4)


@pytest.mark.parametrize("d", [2, 3])
def test_frame_indifference(d):
    F = _rand_F(4, d, 0.2, 31)
    mu, lam = np.full(4, 1.0), np.full(4, 4.0)
    R = O.rotation_matrix([1, 2, 3], 0.7, d)
    RF = np.einsum("ab,pbc->pac", R, F)
    np.testing.assert_allclose(O.psi(RF, mu, lam), O.psi(F, mu, lam), rtol=1e-12)
    np.testing.assert_allclose(O.pk1(RF, mu, lam), np.einsum("ab,pbc->pac", R, O.pk1(F, mu, lam)),
                               atol=1e-12)


def test_inverted_element_has_infinite_energy():
    F = np.array([[[1.0, 0.0], [0.0, -0.5]]])
    assert np.isinf(O.psi(F, np.ones(1), np.ones(1)))[0]


def _problem(dim=2, seed=0, dt=1e-2, E=1e5):
    spec = W.perturb(W.jitter_positions(W.block(dim, n_cells=(4, 3, 3), dx=0.1, E=E,
                                                 gravity=(0.3, -9.8, 0.5)[:dim]), seed), seed + 1)
    gf = O.p2g(spec.particles, spec.grid)
    mask, vel = O.dirichlet_nodes(spec.grid, [], dt)
    return O.make_problem(spec.particles, spec.grid, gf, dt, spec.gravity, mask, vel)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_matches_energy_fd(dim):
    pr = _problem(dim)
    rng = np.random.default_rng(5)
    u = O.initial_guess(pr) + 1e-3 * rng.standard_normal((pr.grid.n_nodes, dim)) * pr.gf.active[:, None]
    g = O.gradient(pr, u)
    act = np.nonzero(pr.gf.active)[0]
    h = 1e-7
    for i in act[:: max(1, act.size // 12)]:
        for a in range(dim):
            e = np.zeros_like(u)
            e[i, a] = h
            fd = (O.energy(pr, u + e) - O.energy(pr, u - e)) / (2 * h)
            np.testing.assert_allclose(g[i, a], fd, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("dim", [2, 3])
def test_hessian_matches_gradient_fd(dim):
    pr = _problem(dim, seed=3)
    rng = np.random.default_rng(6)
    u = O.initial_guess(pr) + 1e-3 * rng.standard_normal((pr.grid.n_nodes, dim)) * pr.gf.active[:, None]
    H = O.hessian(pr, u)
    d = rng.standard_normal(u.shape) * pr.gf.active[:, None]
    Hd = (H @ d.reshape(-1)).reshape(u.shape)
    h = 1e-6
    fd = (O.gradient(pr, u + h * d) - O.gradient(pr, u - h * d)) / (2 * h)
    np.testing.assert_allclose(Hd, fd, rtol=1e-6, atol=1e-4 * np.abs(Hd).max())
    # symmetric
    assert abs(H - H.T).max() <= 1e-9 * abs(H).max()


def test_energy_change_equals_difference():
    pr = _problem(2, seed=8)
    rng = np.random.default_rng(2)
    u = O.initial_guess(pr)
    s = 1e-2 * rng.standard_normal(u.shape) * pr.gf.active[:, None]
    for alpha in (1.0, 0.25):
        np.testing.assert_allclose(O.energy_change(pr, u, s, alpha),
                                   O.energy(pr, u + alpha * s) - O.energy(pr, u), rtol=1e-9)


def test_free_flight_is_exact():
    """Uniform velocity, B = 0, no gravity, no walls: the step is a rigid
    translation (one Newton iteration, F stays I, x += dt v)."""
    spec = W.block(2, n_cells=(4, 3), dx=0.1)
    spec.particles.v[:] = np.array([0.3, -0.2])
    ds = O.DomainState.create(spec)
    ns = O.NewtonStats()
    x0 = ds.p.x.copy()
    O.step(ds, 0.01, ns)
    assert ns.iters == 1
    np.testing.assert_allclose(ds.p.x, x0 + 0.01 * np.array([0.3, -0.2]), atol=1e-15)
    np.testing.assert_allclose(ds.p.F, np.broadcast_to(np.eye(2), ds.p.F.shape), atol=1e-14)
    np.testing.assert_allclose(ds.p.v, np.broadcast_to([0.3, -0.2], ds.p.v.shape), atol=1e-14)


def test_zero_stiffness_free_fall():
    """With a vanishing modulus each node falls freely: v^{n+1} = v^n + dt g."""
    spec = W.block(2, n_cells=(3, 3), dx=0.1, E=1e-12, gravity=(0.0, -9.81))
    ds = O.DomainState.create(spec)
    O.step(ds, 0.01)
    np.testing.assert_allclose(ds.p.v[:, 1], -9.81 * 0.01, rtol=1e-9)
    np.testing.assert_allclose(ds.p.v[:, 0], 0.0, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_prescribed_affine_deformation_is_uniform(dim):
    """Nodes within two cells of the material's edge follow the affine map
    (F_t - I)(x - x0); at a quasi-static step (huge dt) the interior nodes
    follow it too and every particle gets F = F_t (Newton on the nonlinear
    law, checked against the prescribed value)."""
    spec = W.block(dim, n_cells=(8, 8, 6), dx=0.1, E=1e5)
    g = spec.grid
    Ft = np.eye(dim)
    Ft[0, 0], Ft[dim - 1, dim - 1] = 1.02, 0.97
    Ft[0, 1] = 0.01
    xi = O.node_positions(g)
    lo = np.zeros(dim) + 1.5 * g.dx
    hi = np.array([8, 8, 6][:dim]) * g.dx - 1.5 * g.dx
    interior = np.all((xi > lo) & (xi < hi), axis=1)
    dt = 1e3
    vel = (xi @ (Ft - np.eye(dim)).T) / dt
    ds = O.DomainState.create(spec)
    gf = O.p2g(ds.p, g)
    u = O.solve_domain(ds, gf, dt, ~interior, vel)
    np.testing.assert_allclose(u[gf.active], (xi @ (Ft - np.eye(dim)).T)[gf.active], atol=1e-8)
    ds.p = O.g2p(ds.p, g, u, dt)
    np.testing.assert_allclose(ds.p.F, np.broadcast_to(Ft, ds.p.F.shape), atol=1e-8)


def test_newton_reports_exhausted_iterations():
    spec = W.perturb(W.block(2, n_cells=(3, 3), dx=0.1), 1)
    spec = dataclasses.replace(spec, newton_max=1, newton_tol=1e-30)
    ds = O.DomainState.create(spec)
    with pytest.raises(O.NewtonMaxIter):
        O.step(ds, 0.01)


def test_cantilever_first_step_sags():
    spec = W.cantilever()
    ds = O.DomainState.create(spec)
    x0 = ds.p.x.copy()
    O.step(ds, 1e-3)
    dy = ds.p.x[:, 1] - x0[:, 1]
    # free end falls, clamped end barely moves; first step of free fall is g dt^2
    assert dy[x0[:, 0] > 0.9].mean() < 0
    np.testing.assert_allclose(dy[x0[:, 0] > 0.5].mean(), -9.81e-6, rtol=0.05)
    assert abs(dy[x0[:, 0] < 0.0125]).max() < 0.5 * 9.81e-6


@pytest.mark.parametrize("d", [2, 3])
def test_psi_change_identities(d):
    """psi_change equals the plain difference for sizeable dF and the first-
    order term P:dF for tiny dF (where the plain difference is all
    round-off), and reports inversion."""
    F0 = _rand_F(6, d, 0.1, 41 + d)
    mu, lam = np.full(6, 1.7), np.full(6, 2.9)
    rng = np.random.default_rng(4)
    dF = 0.05 * rng.standard_normal((6, d, d))
    np.testing.assert_allclose(O.psi_change(F0, dF, mu, lam),
                               O.psi(F0 + dF, mu, lam) - O.psi(F0, mu, lam), rtol=1e-10)
    tiny = 1e-12 * rng.standard_normal((6, d, d))
    lin = np.sum(O.pk1(F0, mu, lam) * tiny, axis=(1, 2))
    np.testing.assert_allclose(O.psi_change(F0, tiny, mu, lam), lin, rtol=1e-9)
    flip = -2.5 * F0
    assert np.all(np.isinf(O.psi_change(F0, flip, mu, lam)[np.linalg.det(F0 + flip) <= 0]))


def test_round_off_weight_nodes_are_inactive():
    """A particle at a half-cell offset touches the far nodes of its support
    with weight (fx - 1/2)^2 / 2 ~ 1e-32 through rounding; those nodes carry
    no DOF, and the step converges."""
    spec = W.block(2, n_cells=(1, 1), dx=0.1, ppc_1d=1, gravity=(0.0, -9.81))
    gf = O.p2g(spec.particles, spec.grid, mass_eps=spec.mass_eps)
    assert gf.active.sum() == 4
    assert (O.p2g(spec.particles, spec.grid).active.sum()) == 9
    ds = O.DomainState.create(spec)
    O.step(ds, 0.01)
    np.testing.assert_allclose(ds.p.v[:, 1], -9.81 * 0.01, rtol=1e-12)


def _free_problem(spec, dt):
    gf = O.p2g(spec.particles, spec.grid, mass_eps=spec.mass_eps)
    mask, vel = O.dirichlet_nodes(spec.grid, [], dt)
    return O.make_problem(spec.particles, spec.grid, gf, dt, spec.gravity, mask, vel)


def test_initial_guess_takes_the_lower_energy_start():
    """Rigid translation: x_tilde = x^n + dt v^n has zero inertia and no
    strain, so it is the start.  A uniform stretching rate v = c (x - x_c)
    over a step far above the elastic period: x_tilde stretches the block by
    1 + c dt = 6, whose stored energy V E O(1) far exceeds the kinetic term
    m |v|^2 / 2 it saves, so the start is x^n (u = 0 on the free DOFs)."""
    spec = W.block(2, n_cells=(4, 3), dx=0.1, E=1e5)
    spec.particles.v[:] = np.array([0.3, -0.2])
    pr = _free_problem(spec, 0.01)
    u = O.initial_guess(pr)
    a = pr.gf.active
    np.testing.assert_allclose(u[a], np.broadcast_to(0.01 * np.array([0.3, -0.2]), u[a].shape),
                               atol=1e-15)
    spec = W.block(2, n_cells=(4, 3), dx=0.1, E=1e5)
    xc = spec.particles.x.mean(axis=0)
    spec.particles.v[:] = 0.5 * (spec.particles.x - xc)
    pr = _free_problem(spec, 10.0)
    u_tilde = np.where(pr.gf.active[:, None], pr.dt * pr.gf.vn, 0.0)
    assert O.energy_change(pr, np.zeros_like(u_tilde), u_tilde, 1.0) > 0.0
    np.testing.assert_array_equal(O.initial_guess(pr), 0.0)
    # the same field over a short step: x_tilde is the start again
    pr = _free_problem(spec, 1e-3)
    u = O.initial_guess(pr)
    np.testing.assert_allclose(u[a], (pr.dt * pr.gf.vn)[a], rtol=0, atol=0)


@pytest.mark.parametrize("d", [2, 3])
def test_cauchy_stress_from_the_energy(d):
    """sigma = (d psi / d F) F^T / J, with d psi / d F taken by central
    differences of psi (pinned above), not through pk1; symmetric (balance
    of angular momentum), and -p I under a pure volume change with
    p = -(lam ln J + mu (s^2 - 1)) / J for F = s I."""
    F = _rand_F(4, d, 0.15, 11 + d)
    mu, lam = np.full(4, 3.0e5), np.full(4, 7.0e5)
    h = 1e-6
    P = np.zeros_like(F)
    for a in range(d):
        for b in range(d):
            E = np.zeros((d, d))
            E[a, b] = h
            P[:, a, b] = (O.psi(F + E, mu, lam) - O.psi(F - E, mu, lam)) / (2 * h)
    J = np.linalg.det(F)
    sig_fd = np.einsum("pab,pcb->pac", P, F) / J[:, None, None]
    sig = O.cauchy_stress(F, mu, lam)
    np.testing.assert_allclose(sig, sig_fd, rtol=0, atol=1e-6 * np.abs(sig).max())
    np.testing.assert_allclose(sig, np.swapaxes(sig, 1, 2), atol=1e-9 * np.abs(sig).max())
    s = 1.02
    Fs = np.broadcast_to(s * np.eye(d), (1, d, d)).copy()
    Js = s ** d
    p = -(7.0e5 * np.log(Js) + 3.0e5 * (s * s - 1.0)) / Js
    np.testing.assert_allclose(O.cauchy_stress(Fs, mu[:1], lam[:1])[0], -p * np.eye(d),
                               rtol=1e-12, atol=1e-9 * abs(p))


def test_newton_reports_a_failed_line_search(monkeypatch):
    """A line search that finds no decrease within its halving cap is an
    error (LineSearchFailed), not a silently accepted step: forced by
    reporting every trial step as an energy increase."""
    spec = W.cantilever()
    gf = O.p2g(spec.particles, spec.grid, mass_eps=spec.mass_eps)
    mask, vel = O.dirichlet_nodes(spec.grid, spec.dirichlet, 1e-3)
    pr = O.make_problem(spec.particles, spec.grid, gf, 1e-3, spec.gravity, mask, vel)
    calls = []
    monkeypatch.setattr(O, "energy_change", lambda *a: calls.append(a[3]) or 1.0)
    with pytest.raises(O.LineSearchFailed):
        O.newton(pr, spec.newton_tol, spec.newton_max, 3)
    # the cold start compares x_tilde with x^n once, then alpha = 1 and three halvings
    assert calls == [1.0, 1.0, 0.5, 0.25, 0.125]
