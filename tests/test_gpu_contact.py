"""The rigid-plane Hertz benchmark of Sec. 4.2 on the GPU: the unilateral,
gap-aware frictionless plane (osmpm_set_plane; the oracle's reading in
oracle.contact) under the half-cylinder of workloads.hertz_rigid_single,
pressed by its flat face and settled with kinetically damped steps.  The
settled state is compared with the FP64 oracle's stored run of the same
protocol, and its contact pressure with the Hertz semi-ellipse."""
import dataclasses
import os

import numpy as np
import pytest

from oracle import analytic as A
from paper_2605_09097_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DX, PPC_1D, INDENT = 1.0 / 32, 4, 0.03


@pytest.fixture(scope="module")
def osmpm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm as m
    return m


def settle(osmpm, dx, ppc_1d, indent, n_steps=10, dt=0.02, dt_settle=0.2, max_settle=200):
    """The protocol of oracle.contact.settle_hertz through the library: push
    rows following the face down, v and B zeroed after every step, settled
    until the largest particle speed is below 1e-6.  Returns (spec, domain,
    settle steps, contact active sets of the last step)."""
    spec, plane = W.hertz_rigid_single(dx=dx, ppc_1d=ppc_1d, indent=indent, n_steps=n_steps, dt=dt)
    dom = osmpm.Domain(spec)
    dom.set_plane(level=0.0, cand_hi=0.5 * dx, spacing=dx / ppc_1d)
    push = spec.dirichlet[0]

    def damp():
        x, v, B, F = dom.get_particles()
        dom.set_particles(x, np.zeros_like(v), np.zeros_like(B), F)
        return np.abs(v).max()

    for k in range(n_steps):
        lo = (push.lo[0], push.lo[1] - k * indent / n_steps)
        dom.set_dirichlet([dataclasses.replace(push, lo=lo)])
        dom.step(dt)
        damp()
    lo = (push.lo[0], push.lo[1] - indent)
    dom.set_dirichlet([dataclasses.replace(push, lo=lo, vel=(0.0, 0.0, 0.0))])
    for k in range(max_settle):
        st = dom.step(dt_settle)
        if damp() < 1e-6:
            return spec, dom, k + 1, st["contact_sets"]
    raise AssertionError("the contact did not settle")


def _pressure(spec, dom):
    g = spec.grid
    lam = dom.get_grid(osmpm_mod().OSMPM_FIELD_PLANE_FORCE)
    held = dom.get_grid(osmpm_mod().OSMPM_FIELD_PLANE_ACTIVE)
    ix = np.arange(g.res[0] * g.res[1]) % g.res[0]
    p = np.bincount(ix, weights=lam, minlength=g.res[0]) / g.dx
    return p, np.bincount(ix, weights=held, minlength=g.res[0]).astype(int), lam, held


def osmpm_mod():
    from paper_2605_09097_gb300 import osmpm as m
    return m


def _stored():
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_runs",
                        "hertz_rigid_dx1_32_settled.txt")
    p, held, xs, ids, k = [], [], [], [], None
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "settle_steps":
                k = int(parts[1])
            elif parts[0] == "p":
                p.append(float(parts[2]))
                held.append(int(parts[3]))
            elif parts[0] == "x":
                ids.append(int(parts[1]))
                xs.append([float(parts[2]), float(parts[3])])
    return np.asarray(p), np.asarray(held), np.asarray(ids), np.asarray(xs), k


def test_rigid_plane_hertz_matches_oracle_and_hertz(osmpm):
    """Settled GPU contact at dx = 1/32 (16 particles per cell, indent
    0.03): the same settle-step count, held nodes per column and contact
    pressure per column (rel-L2 1e-5) as the oracle's stored run, particle
    displacement within rel-L2 1e-6; the Signorini conditions hold; the
    pressure follows the Hertz semi-ellipse for the transmitted load (edge
    within two node spacings of b, rel-L2 < 0.2) and is symmetric."""
    spec, dom, k, sets = settle(osmpm, DX, PPC_1D, INDENT)
    p, held, lam, act = _pressure(spec, dom)
    op, oheld, ids, ox, ok = _stored()
    assert k == ok
    np.testing.assert_array_equal(held, oheld)
    assert np.linalg.norm(p - op) <= 1e-5 * np.linalg.norm(op)
    x = dom.get_particles()[0][ids]
    x0 = spec.particles.x[ids]
    assert np.linalg.norm(x - ox) <= 1e-6 * np.linalg.norm(ox - x0)
    # Signorini: held nodes push (lambda >= 0), free candidates do not penetrate
    gap = dom.get_grid(osmpm.OSMPM_FIELD_PLANE_GAP)
    u = dom.get_grid(osmpm.OSMPM_FIELD_U)
    assert (lam[act > 0] >= 0.0).all()
    free = np.isfinite(gap) & (act == 0)
    assert (u[free, 1] >= -gap[free] - 1e-12).all()
    # Hertz
    g = spec.grid
    xc = g.origin[0] + np.arange(g.res[0]) * g.dx
    F = p.sum() * g.dx
    b, pmax = A.hertz_line_contact(F, 0.5, 2e5, 0.3)
    edge = np.abs(xc[p > 0]).max()
    assert abs(edge - b) <= 2 * g.dx
    ph = pmax * np.sqrt(np.clip(1.0 - (xc / b) ** 2, 0.0, None))
    sel = np.abs(xc) <= 1.5 * b
    assert np.linalg.norm(p[sel] - ph[sel]) / np.linalg.norm(ph[sel]) < 0.2
    np.testing.assert_allclose(p, p[::-1], rtol=1e-6, atol=1e-9 * pmax)


def test_plane_argument_checks(osmpm):
    spec, _ = W.hertz_rigid_single(dx=1.0 / 16, ppc_1d=2)
    dom = osmpm.Domain(spec)
    with pytest.raises(osmpm.OsmpmError) as e:
        dom.set_plane(level=0.0, cand_hi=0.0, spacing=0.0)
    assert e.value.status == osmpm.OSMPM_E_INVALID
    b3 = osmpm.Domain(W.block(3, n_cells=(3, 3, 3), dx=0.1))
    with pytest.raises(osmpm.OsmpmError) as e:
        b3.set_plane(level=0.0, cand_hi=0.0, spacing=0.05)
    assert e.value.status == osmpm.OSMPM_E_UNSUPPORTED
    dom.set_plane(level=0.0, cand_hi=0.5 / 16, spacing=1.0 / 32)
    cB, cS, sch, dT = W.inclusion(dx_S=0.02, M=2)
    B = osmpm.Domain(cB)
    B.set_plane(level=0.0, cand_hi=0.0, spacing=0.01)
    S = osmpm.Domain(cS)
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.osmpm_schwarz_couple(B, S, dT, sch)
    assert e.value.status == osmpm.OSMPM_E_UNSUPPORTED
