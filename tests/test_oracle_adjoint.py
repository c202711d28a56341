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
