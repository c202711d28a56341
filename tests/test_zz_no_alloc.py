"""The allocation-free energy change (osmpm_energy_change_noalloc) against
the FP64 oracle's energy change and the library's regular entry point for
the same quantity.

It serves callers that may not allocate device memory; its scratch is a
fixed device array, so this test checks two calls in a row (the second call
must not see the first call's leftovers), the size limit and a particle
outside the grid box.  The file is named to be collected last."""
import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-9  # the tolerance of the energy-change parity tests


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm
    return torch, osmpm


def _views(torch, osmpm, spec, m, vn, u, s):
    g, p = spec.grid, spec.particles
    D, n = g.dim, p.n
    dev = "cuda"

    def t(a):
        return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    E, nu = p.E, p.nu
    keep = [t(p.x.T), t(p.F.reshape(n, D * D).T), t(p.vol0), t(E / (2.0 * (1.0 + nu))),
            t(E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))), t(m), t(vn.T), t(u.T), t(s.T)]
    grid = osmpm.osmpm_noalloc_grid()
    grid.dim = D
    for a in range(3):
        grid.origin[a] = g.origin[a] if a < D else 0.0
        grid.res[a] = g.res[a] if a < D else 1
        grid.gravity[a] = spec.gravity[a] if a < D else 0.0
    grid.dx = g.dx
    grid.mass_eps = spec.mass_eps
    grid.m, grid.vn, grid.u, grid.s = (keep[5].data_ptr(), keep[6].data_ptr(),
                                       keep[7].data_ptr(), keep[8].data_ptr())
    parts = osmpm.osmpm_noalloc_particles(n, *(k.data_ptr() for k in keep[:5]))
    return grid, parts, keep


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_energy_change_matches_entry_point(env, dim):
    torch, osmpm = env
    spec = W.perturb(W.jitter_positions(W.block(dim, n_cells=(7, 5, 4), dx=0.1, E=1e5,
                                                 gravity=(0.3, -9.8, 0.2)[:dim]), 21), 22)
    dt = 0.01
    dom = osmpm.Domain(spec)
    nn = spec.grid.n_nodes
    rng = np.random.default_rng(23)
    u = 1e-4 * rng.standard_normal((nn, dim))
    s = 1e-4 * rng.standard_normal((nn, dim))
    ref = [dom.probe_energy_change(dt, u, s, a) for a in (1.0, 0.5)]
    # the oracle on the same grid fields (its own P2G)
    gf = O.p2g(spec.particles, spec.grid, mass_eps=spec.mass_eps)
    mask, vel = O.dirichlet_nodes(spec.grid, [], dt)
    pr = O.make_problem(spec.particles, spec.grid, gf, dt, spec.gravity, mask, vel)
    oracle = [O.energy_change(pr, u, s, a) for a in (1.0, 0.5)]
    grid, parts, keep = _views(torch, osmpm, spec, gf.m, gf.vn, u, s)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for k, alpha in enumerate((1.0, 0.5)):   # two calls in a row on the shared scratch
        st = osmpm.osmpm_energy_change_noalloc(grid, parts, dt, alpha, out.data_ptr() + 8 * k, stream)
        assert st == osmpm.OSMPM_OK, osmpm.osmpm_last_error()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    np.testing.assert_allclose(got, oracle, rtol=RTOL)
    np.testing.assert_allclose(got, ref, rtol=RTOL)


def test_noalloc_reports_a_particle_outside_the_grid(env):
    torch, osmpm = env
    spec = W.perturb(W.block(2, n_cells=(5, 4), dx=0.1, E=1e5), 3)
    nn = spec.grid.n_nodes
    rng = np.random.default_rng(4)
    u = 1e-4 * rng.standard_normal((nn, 2))
    gf = O.p2g(spec.particles, spec.grid, mass_eps=spec.mass_eps)
    grid, parts, keep = _views(torch, osmpm, spec, gf.m, gf.vn, u, u)
    keep[0][0, 3] = spec.grid.origin[0] + 0.2 * spec.grid.dx   # support starts below node 0
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = osmpm.osmpm_energy_change_noalloc(grid, parts, 0.01, 1.0, out.data_ptr(), stream)
    assert st == osmpm.OSMPM_E_OUT_OF_GRID, osmpm.osmpm_last_error()
    assert np.isnan(out.item())
    keep[0][0, 3] = float(spec.particles.x[3, 0])               # back inside: a clean call
    st = osmpm.osmpm_energy_change_noalloc(grid, parts, 0.01, 1.0, out.data_ptr(), stream)
    assert st == osmpm.OSMPM_OK, osmpm.osmpm_last_error()
    assert np.isfinite(out.item())


def test_noalloc_rejects_oversized_problem(env):
    torch, osmpm = env
    spec = W.block(2, n_cells=(2, 2), dx=0.1)
    nn = spec.grid.n_nodes
    z = np.zeros((nn, 2))
    grid, parts, keep = _views(torch, osmpm, spec, np.zeros(nn), z, z, z)
    parts.n = 1 << 21          # claims more particles than the scratch serves
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = osmpm.osmpm_energy_change_noalloc(grid, parts, 0.01, 1.0, out.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)
    assert st == osmpm.OSMPM_E_INVALID
    assert "too large" in osmpm.osmpm_last_error()
