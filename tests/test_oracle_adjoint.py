"""Pins of the oracle's reverse-mode gradient (oracle/adjoint.py) against
central finite differences of the oracle's forward steps (no GPU): the
derivative of J = c . x_final with respect to each particle's Young's
modulus and to every component of the initial state."""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

TOL_N = 1e-13


def _spec(dim, seed):
    rng = np.random.default_rng(seed)
    n_cells = (4, 3, 2)[:dim]
    g = (0.0, -9.81, 0.0)[:dim]
    spec = W.perturb(W.block(dim, n_cells=n_cells, dx=0.1, E=1e5, gravity=g), seed,
                     v_scale=0.2, B_scale=0.01, F_scale=0.02)
    spec.particles.E = spec.particles.E * (1.0 + 0.5 * rng.random(spec.particles.E.shape))
    clamp = W.Dirichlet(lo=(-W.BIG,) * dim, hi=(0.05,) + (W.BIG,) * (dim - 1), comp_mask=(1 << dim) - 1)
    return dataclasses.replace(spec, dirichlet=[clamp]), rng


def _J(spec, dt, n_steps, c):
    ds = O.DomainState.create(spec)
    for _ in range(n_steps):
        AD.record_step(ds, dt, TOL_N)
    return float(np.sum(c * ds.p.x))


def _perturbed(spec, field, index, h):
    p = spec.particles.copy()
    arr = getattr(p, field)
    arr[index] += h
    return dataclasses.replace(spec, particles=p)


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_matches_central_differences(dim):
    spec, rng = _spec(dim, 11 + dim)
    dt, n_steps = 0.01, 2
    n = spec.particles.x.shape[0]
    c = rng.standard_normal((n, dim))
    _, E_bar, bar = AD.trajectory_gradient(spec, dt, n_steps, c, newton_tol=TOL_N)
    assert np.abs(E_bar).max() > 0
    picks = rng.choice(n, 4, replace=False)
    # Young's moduli
    for p in picks:
        h = 1e-4 * spec.particles.E[p]
        fd = (_J(_perturbed(spec, "E", p, h), dt, n_steps, c)
              - _J(_perturbed(spec, "E", p, -h), dt, n_steps, c)) / (2 * h)
        np.testing.assert_allclose(E_bar[p], fd, rtol=1e-5, atol=1e-7 * np.abs(E_bar).max())
    # initial state: positions, velocities, affine matrices, deformation gradients
    cases = [("x", bar.x, 1e-6), ("v", bar.v, 1e-5), ("B", bar.B, 1e-5), ("F", bar.F, 1e-6)]
    for field, adj, h in cases:
        scale = np.abs(adj).max()
        for p in picks:
            comp = tuple(rng.integers(0, dim, size=adj.ndim - 1))
            index = (p,) + comp
            fd = (_J(_perturbed(spec, field, index, h), dt, n_steps, c)
                  - _J(_perturbed(spec, field, index, -h), dt, n_steps, c)) / (2 * h)
            np.testing.assert_allclose(adj[index], fd, rtol=1e-5, atol=1e-6 * scale,
                                       err_msg=f"{field}{index}")


def test_stencil_hessian_matches_differences_of_gradients():
    spec, rng = _spec(2, 5)
    grid = spec.grid
    x = spec.particles.x + 0.013 * rng.standard_normal(spec.particles.x.shape)
    st = O.stencil(x, grid)
    H = AD.stencil_hessian(x, grid, st)
    h = 1e-7
    for b in range(2):
        xp, xm = x.copy(), x.copy()
        xp[:, b] += h
        xm[:, b] -= h
        sp_, sm_ = O.stencil(xp, grid), O.stencil(xm, grid)
        same = np.all(sp_.base == st.base, axis=1) & np.all(sm_.base == st.base, axis=1)
        fd = (sp_.dN - sm_.dN) / (2 * h)
        np.testing.assert_allclose(H[same, :, :, b], fd[same], atol=1e-5 / grid.dx ** 2)
    # symmetric, and the Hessians of a partition of unity sum to zero
    np.testing.assert_allclose(H, H.transpose(0, 1, 3, 2), atol=0)
    np.testing.assert_allclose(H.sum(axis=1), 0.0, atol=1e-10 / grid.dx ** 2)


def _coupled_case():
    """A small coupled inclusion (coarse 0.1, fine 0.05, M = 2) with seeded
    particle velocities, so that every term of the coupled step is live."""
    cB, cS, sch, dT = W.inclusion(dx_S=0.05, dx_B=0.1, M=2, E_inc=4e6)
    rng = np.random.default_rng(3)
    out = []
    for spec in (cB, cS):
        p = spec.particles.copy()
        p.v = 0.01 * rng.standard_normal(p.v.shape)
        p.E = p.E * (1.0 + 0.2 * rng.random(p.E.shape))
        out.append(dataclasses.replace(spec, particles=p))
    return out[0], out[1], sch, dT, rng


def test_recorded_coupled_step_is_schwarz_step():
    cB, cS, sch, dT, _ = _coupled_case()
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    B2, S2 = O.DomainState.create(cB), O.DomainState.create(cS)
    rec = AD.record_schwarz_step(B, S, dT, sch)
    st = O.SchwarzStats()
    O.schwarz_step(B2, S2, dT, sch, st)
    assert len(rec.iters) == st.iters
    np.testing.assert_array_equal(B.p.x, B2.p.x)
    np.testing.assert_array_equal(S.p.F, S2.p.F)


def test_coupled_adjoint_matches_central_differences():
    """Alg. 1 differentiated through the iterations it ran: dJ/dE and the
    start-state adjoints of both particle sets against central differences
    (which run the same number of Schwarz iterations)."""
    cB, cS, sch, dT, rng = _coupled_case()
    nB, nS = cB.particles.n, cS.particles.n
    cb, cs = rng.standard_normal((nB, 2)), rng.standard_normal((nS, 2))

    def J(specB, specS):
        B, S = O.DomainState.create(specB), O.DomainState.create(specS)
        r = AD.record_schwarz_step(B, S, dT, sch, 1e-11)
        return float(np.sum(cb * B.p.x) + np.sum(cs * S.p.x)), len(r.iters)

    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    rec = AD.record_schwarz_step(B, S, dT, sch, 1e-11)
    z = lambda n: (np.zeros((n, 2)), np.zeros((n, 2, 2)), np.zeros((n, 2, 2)))
    vb, Bb, Fb = z(nB)
    vs, Bs, Fs = z(nS)
    B0b, S0b, EB, ES = AD.schwarz_adjoint(rec, AD.StateBar(cb, vb, Bb, Fb), AD.StateBar(cs, vs, Bs, Fs))
    assert len(rec.iters) >= 3 and rec.sets.recvB.sum() > 0 and rec.sets.recvS.sum() > 0
    for which, spec, E_ad, bar in (("B", cB, EB, B0b), ("S", cS, ES, S0b)):
        n = spec.particles.n
        cases = [("E", E_ad, None), ("x", bar.x, 1e-7), ("v", bar.v, 1e-6), ("B", bar.B, 1e-6),
                 ("F", bar.F, 1e-6)]
        for field, adj, h in cases:
            p = int(rng.integers(0, n))
            idx = (p,) + tuple(rng.integers(0, 2, size=adj.ndim - 1))
            hh = 1e-4 * spec.particles.E[p] if field == "E" else h
            vals = []
            for sgn in (1.0, -1.0):
                q = spec.particles.copy()
                getattr(q, field)[idx] += sgn * hh
                s2 = dataclasses.replace(spec, particles=q)
                vals.append(J(s2, cS) if which == "B" else J(cB, s2))
            assert vals[0][1] == vals[1][1] == len(rec.iters)
            fd = (vals[0][0] - vals[1][0]) / (2 * hh)
            np.testing.assert_allclose(adj[idx], fd, rtol=1e-4, atol=1e-5 * np.abs(adj).max(),
                                       err_msg=f"{which} {field}{idx}")
