"""Expanding background of the paper's Test 2 (arXiv 2311.01492, Sec. 4.1.2).

TEST INFRASTRUCTURE (like the rest of ``oracle/``): only ``tests/`` use it.

The test's analytic I-front follows a matter-dominated (Einstein-de Sitter)
expansion, a ∝ t^(2/3), so the proper hydrogen density falls as n_H(t) =
n_H,i (t_i/t)^2 while the grid, the source and the I-front radius are
comoving (a_i = 1 at the ignition time t_i).

* ``age_eds(z, h, omega_m)``: cosmic time at redshift z of that expansion,
  t = 2 / (3 H0 sqrt(Omega_M)) (1 + z)^(-3/2).
* ``scale_factor(t, t_i)``: a(t) = (t / t_i)^(2/3), unity at ignition.
* ``y_closed_form(t, t_i, t_rec_i)``: the comoving volume of the H II region in
  units of the initial Stromgren volume, y = (r_I / r_S,i)^3, from the paper's
  closed form with the second-order exponential integral E2:
      y(t) = lam exp(lam t_i / t) [ (t / t_i) E2(lam t_i / t) - E2(lam) ],
  lam = t_i / t_rec,i (E2 from scipy.special.expn, a library primitive).
* ``y_ode(t, t_i, t_rec_i)``: the same quantity from its defining balance,
  dy/dt = (1 - y (t_i / t)^2) / t_rec,i, y(t_i) = 0 (ionising photons per unit
  time = atoms newly ionised + recombinations in the proper volume), integrated
  numerically -- the independent check of the closed form.
* ``stromgren_radius(ndot, n_H, alpha)``: r_S = (3 Ndot / (4 pi alpha n_H^2))^(1/3).
"""
from __future__ import annotations

import math

import numpy as np

KM_PER_MPC = 3.0856775814913673e19  # km in one Mpc


def age_eds(z, h, omega_m):
    """Cosmic time (s) at redshift z for a matter-dominated expansion."""
    H0 = 100.0 * h / KM_PER_MPC  # s^-1
    return 2.0 / (3.0 * H0 * math.sqrt(omega_m)) * (1.0 + z) ** -1.5


def scale_factor(t, t_i):
    """a(t) with a(t_i) = 1, a ∝ t^(2/3)."""
    return (t / t_i) ** (2.0 / 3.0)


def stromgren_radius(ndot, n_H, alpha):
    return (3.0 * ndot / (4.0 * math.pi * alpha * n_H ** 2)) ** (1.0 / 3.0)


def y_closed_form(t, t_i, t_rec_i):
    """(r_I / r_S,i)^3 at time t >= t_i (Sec. 4.1.2)."""
    from scipy.special import expn
    lam = t_i / t_rec_i
    u = lam * t_i / t
    return lam * math.exp(u) * ((t / t_i) * expn(2, u) - expn(2, lam))


def y_ode(t, t_i, t_rec_i, rtol=1e-12):
    """(r_I / r_S,i)^3 from dy/dt = (1 - y (t_i/t)^2) / t_rec,i, y(t_i) = 0."""
    from scipy.integrate import solve_ivp
    if t <= t_i:
        return 0.0
    sol = solve_ivp(lambda s, y: [(1.0 - y[0] * (t_i / s) ** 2) / t_rec_i], (t_i, t), [0.0],
                    method="DOP853", rtol=rtol, atol=1e-16)
    return float(sol.y[0, -1])
