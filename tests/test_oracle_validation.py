"""Validation pins from the paper's closed forms (no GPU): the elastica of
Sec. 4.1 and its Euler-Bernoulli limit, the Hertz and Eshelby formulas of
Sec. 4.2-4.3, and the oracle's quasi-static cantilever against the
elastica (the progressive static solve of Sec. 2.2.6)."""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W


def test_elastica_small_load_is_euler_bernoulli():
    for g in (1e-3, 1e-2):
        np.testing.assert_allclose(A.elastica_tip_deflection(g), g / 8, rtol=2e-3)


def test_elastica_stiffens_geometrically():
    g = 2.0
    assert A.elastica_tip_deflection(g) < g / 8
    s, th, x, y = A.elastica(g)
    np.testing.assert_allclose(np.hypot(np.diff(x), np.diff(y)).sum(), 1.0, rtol=1e-5)  # inextensible


def test_hertz_force_balance():
    F, R = 120.0, 0.5
    b, pmax = A.hertz_line_contact(F, R, 2e5, 0.3)
    x = np.linspace(-b, b, 20001)
    p = pmax * np.sqrt(np.clip(1 - (x / b) ** 2, 0, None))
    np.testing.assert_allclose(np.trapezoid(p, x), F, rtol=1e-4)
    b2, _ = A.hertz_line_contact(F, R, 2e5, 0.3, 2e5, 0.3)        # two equal bodies: E* halves
    np.testing.assert_allclose(b2, b * np.sqrt(2.0), rtol=1e-12)


def test_eshelby_limits():
    G = 1e6 / 2.6
    # rigid inclusion: P -> 2 G_out delta
    np.testing.assert_allclose(A.eshelby_pressure(0.01, 1e15, 0.3, 1e6, 0.3), 2 * G * 0.01, rtol=1e-8)
    # identical materials: P = delta G / (1 - nu)
    np.testing.assert_allclose(A.eshelby_pressure(0.01, 1e6, 0.3, 1e6, 0.3), 0.01 * G / 0.7, rtol=1e-12)
    srr, stt = A.eshelby_stress(np.array([0.5, 2.0]), 1.0, 3.0)
    np.testing.assert_allclose(srr, [-3.0, -0.75])
    np.testing.assert_allclose(stt, [-3.0, 0.75])


def quasi_static_cantilever_tip(gamma, dt=0.5, max_steps=60):
    spec = W.cantilever(g=-W.eb_gravity(gamma))
    ds = O.DomainState.create(spec)
    x0 = spec.particles.x.copy()
    tip = x0[:, 0] > 0.98
    for _ in range(max_steps):
        O.step(ds, dt)
        if np.abs(ds.p.v).max() < 1e-6:
            break
    assert np.abs(ds.p.v).max() < 1e-6
    return -(ds.p.x[tip, 1] - x0[tip, 1]).mean(), ds


@pytest.mark.parametrize("gamma", [0.05, 0.231])
def test_oracle_cantilever_matches_elastica(gamma):
    """The beam [0,1]x[0,0.1] (8 cells thick, 2x2 ppc), clamped at x <= 0,
    settles within 3 % of the elastica tip deflection (MPM's shear and
    clamp smearing add ~1 %)."""
    w, _ = quasi_static_cantilever_tip(gamma)
    np.testing.assert_allclose(w, A.elastica_tip_deflection(gamma), rtol=0.03)


def _settled_hertz_contact(dx, ppc_1d, indent, n_steps=10, dt=0.02, dt_settle=0.2):
    """oracle.contact.settle_hertz without its settle-step count."""
    from oracle import contact as C
    return C.settle_hertz(dx, ppc_1d, indent, n_steps, dt, dt_settle)[:8]


def test_unilateral_plane_contact_gives_the_hertz_pressure():
    """The oracle's reading of the rigid frictionless plane (a gap-aware
    Signorini condition on the plane nodes' normal motion, oracle.contact)
    satisfies the Signorini conditions at the settled state, and its
    contact pressure (plane multipliers summed per node column / dx) follows
    the Hertz semi-ellipse p_max sqrt(1 - (x/b)^2) with b and p_max from
    the transmitted load: half-width within two node spacings, relative L2
    error below 0.2 at dx = 1/32 with 16 particles per cell."""
    dx = 1.0 / 32
    spec, plane, gf, gap, act, lam, u, _ = _settled_hertz_contact(dx, 4, 0.03)
    cand = plane & gf.active & np.isfinite(gap)
    # Signorini: lambda >= 0 where held, no penetration where free
    assert (lam[act] >= 0.0).all()
    assert (u[cand & ~act, 1] >= -gap[cand & ~act] - 1e-12).all()
    g = spec.grid
    ix = np.arange(g.res[0] * g.res[1]) % g.res[0]
    p = np.bincount(ix, weights=np.where(plane, lam, 0.0), minlength=g.res[0]) / dx
    xc = g.origin[0] + np.arange(g.res[0]) * dx
    F = p.sum() * dx
    b, pmax = A.hertz_line_contact(F, 0.5, 2e5, 0.3)
    edge = np.abs(xc[p > 0]).max()
    assert abs(edge - b) <= 2 * dx
    ph = pmax * np.sqrt(np.clip(1.0 - (xc / b) ** 2, 0.0, None))
    sel = np.abs(xc) <= 1.5 * b
    err = np.linalg.norm(p[sel] - ph[sel]) / np.linalg.norm(ph[sel])
    assert err < 0.2, err
    np.testing.assert_allclose(p, p[::-1], rtol=1e-6, atol=1e-9 * pmax)   # symmetric about x = 0
