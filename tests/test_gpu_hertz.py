"""Hertzian contact OS-MPM (elastic half-disk pressed into an elastic
block, fine subdomain around the contact, M = 4).  A reduced-resolution
variant is compared with the FP64 oracle particle by particle, in FP64 and
in mixed precision; the full-size configuration (dx_c 1/64, ~166k
particles, mixed) runs two global steps and is checked through properties
that hold at any size, and run whole against the Hertz closed form."""
import dataclasses

import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = dict(dx_c=1.0 / 8, ratio=2, box_lo=(1.25, 1.5), box_hi=(2.75, 2.5))


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


@pytest.mark.parametrize("precision,tol", [(0, 1e-6), (1, 1e-4)])
def test_hertz_reduced_matches_oracle(osmpm, precision, tol):
    cB, cS, sch, dT = W.hertz(precision=precision, **SMALL)
    assert (cB.particles.flags > 0).sum() > 0 and (cS.particles.flags > 0).sum() > 0
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    oB = O.DomainState.create(dataclasses.replace(cB, precision=0))
    oS = O.DomainState.create(dataclasses.replace(cS, precision=0))
    for _ in range(3):
        st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
        so = {}
        O.schwarz_step(oB, oS, dT, sch, O.SchwarzStats(), so)
        assert st["converged"] == 1
    np.testing.assert_array_equal(B.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0, so["sets"].recvB)
    np.testing.assert_array_equal(S.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0, so["sets"].recvS)
    assert rel_disp(B.get_particles()[0], oB.p.x, cB.particles.x) <= tol
    assert rel_disp(S.get_particles()[0], oS.p.x, cS.particles.x) <= tol


def test_hertz_full_size_two_steps(osmpm):
    cB, cS, sch, dT = W.hertz()          # dx_c 1/64, dx_f 1/256, M = 4, mixed
    assert cB.particles.n + cS.particles.n > 150_000
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    for _ in range(2):
        st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
        assert st["converged"] == 1
    xB, vB, _, FB = B.get_particles()
    xS, vS, _, FS = S.get_particles()
    for a in (xB, vB, FB, xS, vS, FS):
        assert np.all(np.isfinite(a))
    assert np.linalg.det(FB).min() > 0 and np.linalg.det(FS).min() > 0
    # the flat face's grid nodes carry the prescribed displacement exactly; the
    # block bottom stays put
    v_push = -0.02 / (100 * dT)
    u = B.get_grid(osmpm.OSMPM_FIELD_U)
    m = B.get_grid(osmpm.OSMPM_FIELD_MASS)
    ny = cB.grid.res[1]
    yi = cB.grid.origin[1] + cB.grid.dx * (np.arange(cB.grid.n_nodes) // cB.grid.res[0])
    face = (yi >= 2.5 - 0.5 * cB.grid.dx) & (m > cB.mass_eps)
    assert face.sum() > 10
    np.testing.assert_allclose(u[face, 1], v_push * dT, rtol=1e-12)
    np.testing.assert_allclose(u[face, 0], 0.0, atol=1e-15)
    top = cB.particles.x[:, 1] > 2.5 - cB.grid.dx
    assert v_push < vB[top, 1].mean() < 0.5 * v_push
    bottom = cB.particles.x[:, 1] < cB.grid.dx
    assert np.abs(xB[bottom] - cB.particles.x[bottom]).max() < 1e-3 * abs(v_push) * 2 * dT
    # coupled: fine particles in the contact zone move down with the indenter
    near = (np.abs(cS.particles.x[:, 0] - 2.0) < 0.05) & (cS.particles.x[:, 1] > 2.0)
    assert (xS[near, 1] - cS.particles.x[near, 1]).mean() < 0


def test_hertz_full_size_pressure_matches_closed_form(osmpm):
    """The full contact configuration run whole (100 global steps, the flat
    face pushed down 0.02): from step 60 on, once the start-up transient of
    the sudden push has passed, the pressure on the block's top layer, fitted
    by a semi-ellipse, has its half-width b and peak p_max within 15 % of the
    Hertz line contact at the measured load (cylinder on a half-space, plane
    strain).  The configuration bonds the bodies (R22) and loads them
    dynamically, where Hertz assumes frictionless static contact, so the
    bound is an engineering one."""
    import bench
    out = bench.run_hertz(None, 0, 0, 1)
    late = [r for r in out["profiles"] if r["step"] >= 60]
    assert len(late) == 5
    for r in late:
        assert r["F_N_per_m"] > 1e4, r
        assert abs(r["b_fit"] / r["b_hertz"] - 1.0) <= 0.15, r
        assert abs(r["p_max_fit"] / r["p_max_hertz"] - 1.0) <= 0.15, r
