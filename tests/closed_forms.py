"""Closed-form solutions of the paper used as expected values by the tests (no GPU, no oracle).

App. A (one-dimensional phase change, diffuse model), liquid where d > 0 (H = 1), gas where d < 0, inflow u_bar
along the direction from the liquid into the gas:
  u(d) = u_bar + mdot (1 - H(d)) (1/rho_g - 1/rho_l)          Eq. (stefan_diffuse_velocity)
  p(d) = mdot^2 H(d) (1/rho_g - 1/rho_l)                       Eq. (stefan_diffuse_pressure), zero at the gas outlet
with the smoothed Heaviside of the signed distance, Eq. (heaviside):
  H = 0 (d <= -3 eps), 1/2 + d/(6 eps) + sin(pi d / (3 eps)) / (2 pi) (|d| < 3 eps), 1 (d >= 3 eps).
The interface is static when u_bar = mdot / rho_l (Eq. 1DStefan_uGamma_sharp).
"""
from __future__ import annotations

import math

import numpy as np


def heaviside_of_distance(d, eps):
    d = np.asarray(d, dtype=float)
    inner = 0.5 + d / (6.0 * eps) + np.sin(math.pi * d / (3.0 * eps)) / (2.0 * math.pi)
    return np.where(d >= 3.0 * eps, 1.0, np.where(d <= -3.0 * eps, 0.0, inner))


def stefan_diffuse(d, eps, mdot, rho_l, rho_g, u_bar=None):
    """(u, p) of the diffuse 1D phase change at signed distances d; u_bar defaults to the static inflow mdot/rho_l."""
    if u_bar is None:
        u_bar = mdot / rho_l
    H = heaviside_of_distance(d, eps)
    jump = 1.0 / rho_g - 1.0 / rho_l
    return u_bar + mdot * (1.0 - H) * jump, mdot * mdot * H * jump
