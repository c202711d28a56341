"""Closed-form and ODE references of the paper's validation problems.

TEST INFRASTRUCTURE ONLY (imported by the tests, never by the library).

* Planar elastica of a clamped-free beam under its own weight (Sec. 4.1):
  theta'' + Gamma (1 - s) cos(theta) = 0, theta(0) = 0, theta'(1) = 0,
  x' = cos(theta), y' = sin(theta), with Gamma the gravito-bending number
  rho g A L^3 / (D w).  Its small-Gamma limit is Euler-Bernoulli:
  tip deflection / L = Gamma / 8.
* Hertz line contact (Sec. 4.2): half-width b = 2 sqrt(F R / (pi E*)),
  p_max = 2 F / (pi b), 1/E* = (1 - nu1^2)/E1 + (1 - nu2^2)/E2 (the paper's
  rigid-plane case is E2 -> infinity).
* Eshelby inclusion under a uniform eigenstrain in plane strain (Sec. 4.3):
  interface pressure P = delta / (C_out + C_in), C_out = 1/(2 G_out),
  C_in = (1 - 2 nu_in)/(2 G_in); inside sigma_rr = sigma_tt = -P; outside
  sigma_rr = -P (R/r)^2, sigma_tt = +P (R/r)^2.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq


def elastica(gamma: float, n: int = 401):
    """Shape of the gravity-loaded elastica: returns (s, theta, x, y), found
    by shooting on theta'(0) so that theta'(1) = 0.  In this form theta >= 0
    and y >= 0 is the deflection in the direction of the load."""

    def rhs(s, z):
        th, k, x, y = z
        return [k, -gamma * (1.0 - s) * np.cos(th), np.cos(th), np.sin(th)]

    def miss(k0):
        sol = solve_ivp(rhs, (0.0, 1.0), [0.0, k0, 0.0, 0.0], rtol=1e-12, atol=1e-14)
        return sol.y[1, -1]

    # theta'(1) < 0 at theta'(0) = 0 and > 0 at theta'(0) = gamma
    k0 = brentq(miss, 0.0, gamma, xtol=1e-15)
    s = np.linspace(0.0, 1.0, n)
    sol = solve_ivp(rhs, (0.0, 1.0), [0.0, k0, 0.0, 0.0], t_eval=s, rtol=1e-12, atol=1e-14)
    return s, sol.y[0], sol.y[2], sol.y[3]


def elastica_tip_deflection(gamma: float) -> float:
    """y(1): the tip deflection over L of the elastica."""
    return float(elastica(gamma)[3][-1])


def hertz_line_contact(F: float, R: float, E1: float, nu1: float, E2: float = np.inf,
                       nu2: float = 0.0):
    """(b, p_max) of a cylinder of radius R pressed with force F per unit
    length onto a half-space; E2 = inf is the rigid plane."""
    inv = (1.0 - nu1 ** 2) / E1 + (0.0 if np.isinf(E2) else (1.0 - nu2 ** 2) / E2)
    E_star = 1.0 / inv
    b = 2.0 * np.sqrt(F * R / (np.pi * E_star))
    return b, 2.0 * F / (np.pi * b)


def eshelby_pressure(delta: float, E_in: float, nu_in: float, E_out: float, nu_out: float) -> float:
    """Interface pressure P of a circular inclusion with uniform eigenstrain
    -delta in an infinite plane-strain matrix."""
    G_in = E_in / (2.0 * (1.0 + nu_in))
    G_out = E_out / (2.0 * (1.0 + nu_out))
    C_out = 1.0 / (2.0 * G_out)
    C_in = (1.0 - 2.0 * nu_in) / (2.0 * G_in)
    return delta / (C_out + C_in)


def eshelby_stress(r: np.ndarray, R: float, P: float):
    """(sigma_rr, sigma_tt) at radius r."""
    r = np.asarray(r, dtype=np.float64)
    inside = r < R
    q = np.where(inside, 1.0, (R / np.maximum(r, 1e-300)) ** 2)
    return np.where(inside, -P, -P * q), np.where(inside, -P, P * q)
