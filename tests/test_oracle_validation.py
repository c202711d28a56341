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
