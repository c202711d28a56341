"""Pins of the oracle's shape functions, indexing, Morton order and transfers
against textbook facts (no GPU).  Each test would fail for a plausible typo
in the oracle: a wrong branch of the B-spline, a swapped axis in the flat
index, a transposed B in the APIC transfer, a missing D^-1."""
import os

import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(dim=2, dx=0.1, res=None):
    res = res or ((12, 10) if dim == 2 else (8, 7, 9))
    return W.Grid(dim, tuple([-0.3, -0.2, -0.1][:dim]), dx, tuple(res))


def _random_x(grid, n, seed):
    rng = np.random.default_rng(seed)
    lo = np.asarray(grid.origin) + 2.0 * grid.dx
    hi = np.asarray(grid.origin) + (np.asarray(grid.res) - 3.0) * grid.dx
    return lo + (hi - lo) * rng.random((n, grid.dim))


def test_bspline_golden_values():
    data = np.loadtxt(os.path.join(GOLDEN, "bspline2_values.txt"))
    np.testing.assert_allclose(O.bspline2(data[:, 0]), data[:, 1], rtol=0, atol=1e-15)


def test_bspline_is_threefold_box_convolution():
    # cardinal quadratic B-spline = box * box * box, computed numerically
    h = 1e-4
    s = np.arange(-0.5, 0.5, h) + h / 2
    box = np.ones_like(s)
    tri = np.convolve(box, box) * h
    quad = np.convolve(tri, box) * h
    r = (np.arange(quad.size) - (quad.size - 1) / 2) * h
    np.testing.assert_allclose(O.bspline2(r), quad, atol=5e-4)


def test_bspline_derivative_matches_central_difference():
    r = np.linspace(-1.7, 1.7, 341) + 1e-3
    h = 1e-6
    fd = (O.bspline2(r + h) - O.bspline2(r - h)) / (2 * h)
    np.testing.assert_allclose(O.bspline2_deriv(r), fd, atol=1e-6)


@pytest.mark.parametrize("dim", [2, 3])
def test_partition_of_unity_and_linear_reproduction(dim):
    g = _grid(dim)
    x = _random_x(g, 200, 1 + dim)
    st = O.stencil(x, g)
    np.testing.assert_allclose(st.N.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.einsum("pk,pka->pa", st.N, st.xi), x, atol=1e-14)
    np.testing.assert_allclose(st.dN.sum(1), 0.0, atol=1e-11)
    # sum_i x_i grad N_i^T = I
    G = np.einsum("pka,pkb->pab", st.xi, st.dN)
    np.testing.assert_allclose(G, np.broadcast_to(np.eye(dim), G.shape), atol=1e-12)
    # APIC inertia tensor of the quadratic B-spline: D = dx^2/4 I
    r = st.xi - x[:, None, :]
    D = np.einsum("pk,pka,pkb->pab", st.N, r, r)
    np.testing.assert_allclose(D, np.broadcast_to(g.dx ** 2 / 4 * np.eye(dim), D.shape), atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_stencil_against_brute_force_scan(dim):
    g = _grid(dim)
    x = _random_x(g, 25, 7 + dim)
    st = O.stencil(x, g)
    xi = O.node_positions(g)
    for p in range(x.shape[0]):
        r = (x[p][None, :] - xi) / g.dx
        w = np.prod(O.bspline2(r), axis=1)
        nz = np.nonzero(w > 0)[0]
        got = dict(zip(st.node[p], st.N[p]))
        assert set(nz) <= set(got)
        for i in range(xi.shape[0]):
            np.testing.assert_allclose(got.get(i, 0.0), w[i], atol=1e-15)


def test_flat_index_is_x_fastest():
    g = _grid(2, res=(5, 4))
    xi = O.node_positions(g)
    # node (i, j) has flat index i + 5 j
    np.testing.assert_allclose(xi[1 + 5 * 2], [g.origin[0] + g.dx, g.origin[1] + 2 * g.dx])


def test_morton_golden_4x4():
    table = np.loadtxt(os.path.join(GOLDEN, "morton_4x4.txt"), dtype=np.int64)
    jj, ii = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    base = np.stack([ii.reshape(-1), jj.reshape(-1)], axis=1)
    np.testing.assert_array_equal(O.morton_code(base).reshape(4, 4), table)


def test_morton_3d_unit_bits():
    base = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [2, 0, 0], [0, 0, 4]])
    np.testing.assert_array_equal(O.morton_code(base), [1, 2, 4, 8, 256])


def test_sort_order_is_stable_on_ties():
    g = _grid(2)
    x = np.array([[0.08, 0.08], [0.3, 0.1], [0.09, 0.07], [0.081, 0.079]])
    order = O.sort_order(x, g)
    # particles 0, 2, 3 share a base cell and keep id order
    assert list(order[:3]) == [0, 2, 3]


@pytest.mark.parametrize("dim", [2, 3])
def test_p2g_conserves_mass_momentum_and_angular_momentum(dim):
    spec = W.perturb(W.jitter_positions(W.block(dim, n_cells=(4, 3, 3), dx=0.1), 3), 4)
    p, g = spec.particles, spec.grid
    gf = O.p2g(p, g)
    np.testing.assert_allclose(gf.m.sum(), p.mass.sum(), rtol=1e-14)
    np.testing.assert_allclose(gf.mv.sum(0), (p.mass[:, None] * p.v).sum(0), atol=1e-13)
    xi = O.node_positions(g)
    if dim == 2:
        L_grid = np.sum(xi[:, 0] * gf.mv[:, 1] - xi[:, 1] * gf.mv[:, 0])
        L_part = np.sum(p.mass * (p.x[:, 0] * p.v[:, 1] - p.x[:, 1] * p.v[:, 0]
                                   + p.B[:, 1, 0] - p.B[:, 0, 1]))
        np.testing.assert_allclose(L_grid, L_part, rtol=1e-12)
    else:
        L_grid = np.cross(xi, gf.mv).sum(0)
        eps = np.zeros((3, 3, 3))
        eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
        eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
        L_part = (p.mass[:, None] * (np.cross(p.x, p.v) + np.einsum("cab,pba->pc", eps, p.B))).sum(0)
        np.testing.assert_allclose(L_grid, L_part, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_affine_field_round_trip(dim):
    """G2P of an affine grid velocity a + C x gives v_p = a + C x_p and
    B_p = C D; P2G of that state gives back a + C x_i on active nodes."""
    spec = W.jitter_positions(W.block(dim, n_cells=(4, 3, 3), dx=0.1), 5)
    p, g = spec.particles, spec.grid
    rng = np.random.default_rng(9)
    a = rng.standard_normal(dim)
    C = rng.standard_normal((dim, dim))
    xi = O.node_positions(g)
    dt = 0.01
    u = dt * (a[None] + xi @ C.T)
    q = O.g2p(p, g, u, dt)
    np.testing.assert_allclose(q.v, a[None] + p.x @ C.T, atol=1e-12)
    np.testing.assert_allclose(q.B, np.broadcast_to(C * g.dx ** 2 / 4, q.B.shape), atol=1e-13)
    gf = O.p2g(p.__class__(p.x, q.v, q.B, p.F, p.vol0, p.mass, p.E, p.nu, p.flags), g)
    act = gf.active
    np.testing.assert_allclose(gf.vn[act], a[None] + xi[act] @ C.T, atol=1e-12)


def test_out_of_grid_is_reported():
    g = _grid(2)
    with pytest.raises(O.OutOfGrid):
        O.stencil(np.array([[g.origin[0] + 0.5 * g.dx, 0.3]]), g)
