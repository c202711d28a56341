"""The block-tiled Hessian-vector product of the streaming PCG (mixed
precision, hvp_mode 2): each block stages the grid nodes its Morton-sorted
particles touch in shared memory and recomputes the particle Hessian from
the Newton iterate.  Checked against the oracle's assembled Hessian element
by element, against the lane-group product, and through whole steps; a
configuration whose particles sit in two far-apart clusters makes one block's
node box larger than the tile, which takes the global-memory path."""
import dataclasses

import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def osmpm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm as m
    return m


def rel_disp(x_gpu, x_ref, x0):
    return np.linalg.norm(x_gpu - x_ref) / max(np.linalg.norm(x_ref - x0), 1e-300)


def two_clusters(dim, gap_cells=40):
    """Two blocks of material (6^2 cells in 2D, 4^3 in 3D) at opposite
    corners of a grid whose node box spans gap_cells cells per axis.  In
    Morton order the slot tile that holds the end of the first cluster and
    the start of the second has a node box far larger than the tile (the
    global-memory path); the other tiles are staged in shared memory.  In
    both dimensions the last tile ends inside a warp (a partly filled warp
    of slots)."""
    dx, ppc = 0.05, 2
    c = 6 if dim == 2 else 4
    inside = lambda x: np.ones(len(x), dtype=bool)  # noqa: E731
    a = W.sample_lattice((0.0,) * dim, dx, (0,) * dim, (c,) * dim, ppc, inside)
    b = W.sample_lattice((0.0,) * dim, dx, (gap_cells - c,) * dim, (gap_cells,) * dim, ppc, inside)
    x = np.concatenate([a, b])
    p = W.make_particles(x, dx, ppc, 1000.0, 1e5, 0.3)
    m = 3
    grid = W.Grid(dim, (-m * dx,) * dim, dx, (gap_cells + 2 * m + 1,) * dim)
    g = (0.0, -9.81, 0.0)[:dim]
    return W.DomainSpec(f"two_clusters{dim}d", grid, p, g, [])


def _problem(spec, dt, seed):
    gf = O.p2g(spec.particles, spec.grid, mass_eps=spec.mass_eps)
    mask, vel = O.dirichlet_nodes(spec.grid, [], dt)
    pr = O.make_problem(spec.particles, spec.grid, gf, dt, spec.gravity, mask, vel)
    rng = np.random.default_rng(seed)
    u = O.initial_guess(pr) + 1e-3 * spec.grid.dx * rng.standard_normal(pr.gf.vn.shape) * gf.active[:, None]
    d = rng.standard_normal(u.shape) * gf.active[:, None]
    return pr, u, d


@pytest.mark.parametrize("case", ["block2", "block3", "clusters2", "clusters3"])
@pytest.mark.parametrize("hvp_mode", [1, 2])
def test_streaming_hvp_matches_assembled_hessian(osmpm, case, hvp_mode):
    """(M/dt^2 + K(u)) d from the streaming product in mixed precision
    against the oracle's assembled FP64 Hessian: every component within
    2e-5 of the largest (FP32 arithmetic)."""
    dim = int(case[-1])
    if case.startswith("block"):
        spec = W.perturb(W.jitter_positions(W.block(dim, n_cells=(9, 7, 5), dx=0.1, E=1e5,
                                                    gravity=(0.2, -9.8, 0.1)[:dim]), 3), 4)
    else:
        spec = W.perturb(two_clusters(dim), 5)
    dt = 0.01
    pr, u, d = _problem(spec, dt, 11)
    dom = osmpm.Domain(dataclasses.replace(spec, precision=1, pcg_mode=2, hvp_mode=hvp_mode))
    H = O.hessian(pr, u)
    hd_ref = (H @ d.reshape(-1)).reshape(u.shape) * pr.gf.active[:, None]
    hd = dom.probe_hvp(dt, u, d)
    np.testing.assert_allclose(hd, hd_ref, rtol=0, atol=2e-5 * np.abs(hd_ref).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_tiled_steps_match_oracle(osmpm, dim):
    """Steps through the streaming PCG with the tiled product (mixed) on a
    perturbed block and on the two-cluster configuration: displacement
    within rel-L2 1e-4 of the FP64 oracle; the tiled and the lane-group
    products give the same steps within that tolerance."""
    for spec in (W.perturb(W.block(dim, n_cells=(8, 6, 4), dx=0.1, E=1e5,
                                   gravity=(0.0, -9.8, 0.0)[:dim]), 9),
                 W.perturb(two_clusters(dim), 10)):
        ref = O.DomainState.create(spec)
        doms = {m: osmpm.Domain(dataclasses.replace(spec, precision=1, pcg_mode=2, hvp_mode=m))
                for m in (1, 2)}
        x0 = spec.particles.x.copy()
        for _ in range(5):
            O.step(ref, 0.01)
            for dom in doms.values():
                dom.step(0.01)
        x = {m: dom.get_particles()[0] for m, dom in doms.items()}
        assert rel_disp(x[2], ref.p.x, x0) <= MIXED_TOL, spec.name
        assert rel_disp(x[1], ref.p.x, x0) <= MIXED_TOL, spec.name
        assert rel_disp(x[2], x[1], x0) <= MIXED_TOL, spec.name
