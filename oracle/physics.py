"""Per-point material law of the diffuse-interface model (test infrastructure, see package docstring).

Every function evaluates the paper's formula literally, on arrays of level-set values / gradients:
  distance   d(phi) = eps log((1 + phi) / (1 - phi))                                   Eq. (distance)
  heaviside  H = 0 (d <= -3 eps), 1/2 + d/(6 eps) + sin(pi d / (3 eps)) / (2 pi), 1 (d >= 3 eps)   Eq. (heaviside)
  delta      delta = |grad H(phi)| = H'(d) d'(phi) |grad phi|                          Eq. (delta)
  density    1/rho = H/rho_l + (1 - H)/rho_g  (reciprocal)                             Eq. (rhoEff)
  viscosity  mu = H mu_l + (1 - H) mu_g                                                Eq. (muEff)
  normal     n = grad phi / |grad phi|                                                 Eq. (normal_vector)
  dilation   v = mdot (1/rho_g - 1/rho_l) delta          Eq. (evaporDil), sign of App. A (see dilation_rate)

Reading of the branch boundaries (the paper's cases are in d; d(phi) is increasing): the interface zone
0 < H < 1 is |phi| < tanh(3/2), i.e. -3 eps < d < 3 eps.  Outside it H is 0 or 1, its derivatives vanish and the
logarithm is never evaluated (|phi| may round to 1 there).
"""
from __future__ import annotations

import numpy as np

# phi at d = 3 eps (Eq. initial_phi at d = 3 eps): tanh(3/2) = 0.90514825364486643824..., correctly rounded
# (numpy's tanh(1.5) is one ulp above it).  The zone test |phi| < PHI_BAND decides an integer (inside / outside),
# so it is taken with this exact double.
PHI_BAND = float.fromhex("0x1.cf6f9786df577p-1")
PHI_GAS_BAND = float.fromhex("0x1.fd77d111a0b00p-1")  # tanh(3) correctly rounded (d = 6 eps)


def distance(phi, eps):
    """Signed distance recovered from the regularized level set, Eq. (distance)."""
    phi = np.asarray(phi, dtype=float)
    return eps * np.log((1.0 + phi) / (1.0 - phi))


def in_zone(phi):
    """Interface zone 0 < H < 1 (equivalently -3 eps < d(phi) < 3 eps)."""
    return np.abs(np.asarray(phi, dtype=float)) < PHI_BAND


def heaviside_parts(phi, eps):
    """Returns (H, dH/dd, d^2H/dd^2, d, zone) at every point; derivatives are zero outside the zone."""
    phi = np.asarray(phi, dtype=float)
    zone = in_zone(phi)
    H = np.where(phi >= PHI_BAND, 1.0, 0.0)
    dH = np.zeros_like(phi)
    d2H = np.zeros_like(phi)
    d = np.zeros_like(phi)
    pz = phi[zone]
    dz = distance(pz, eps)
    arg = np.pi * dz / (3.0 * eps)
    H[zone] = 0.5 + dz / (6.0 * eps) + np.sin(arg) / (2.0 * np.pi)
    dH[zone] = (1.0 + np.cos(arg)) / (6.0 * eps)
    d2H[zone] = -np.pi * np.sin(arg) / (18.0 * eps * eps)
    d[zone] = dz
    return H, dH, d2H, d, zone


def heaviside(phi, eps):
    return heaviside_parts(phi, eps)[0]


def ddist_dphi(phi, eps):
    """d'(phi) = 2 eps / (1 - phi^2)."""
    phi = np.asarray(phi, dtype=float)
    return 2.0 * eps / (1.0 - phi * phi)


def d2dist_dphi2(phi, eps):
    """d''(phi) = 4 eps phi / (1 - phi^2)^2."""
    phi = np.asarray(phi, dtype=float)
    return 4.0 * eps * phi / (1.0 - phi * phi) ** 2


def density(H, rho_l, rho_g, mode="reciprocal"):
    """Effective density: reciprocal interpolation Eq. (rhoEff); mode 'arithmetic' is the contrast case of Sec. 3.1."""
    H = np.asarray(H, dtype=float)
    if mode == "arithmetic":
        return H * rho_l + (1.0 - H) * rho_g
    return 1.0 / (H / rho_l + (1.0 - H) / rho_g)


def viscosity(H, mu_l, mu_g):
    """Effective dynamic viscosity, Eq. (muEff)."""
    H = np.asarray(H, dtype=float)
    return H * mu_l + (1.0 - H) * mu_g


GRAD_TINY = 1e-4  # |grad phi| h at or below this: phi varies by < 1e-4 across a cell (> ~9 eps from the interface)


def has_normal(gnorm, h):
    """Where the normal of Eq. (normal_vector) is taken as defined: |grad phi| h > 1e-4.  Reading: where phi has
    saturated towards +-1 (more than ~9 eps from any interface, outside the interface zone and the projection band)
    the direction of grad phi is ill-conditioned (relative error ~ 1e-16 / (|grad phi| h), pure rounding noise where
    phi is exactly +-1) and without physical meaning; n is taken as 0 there."""
    return np.asarray(gnorm) * h > GRAD_TINY


def normal(grad_phi, h):
    """Unit normal of Eq. (normal_vector), grad_phi[..., 3]; zero where the gradient is negligible (has_normal)."""
    g = np.asarray(grad_phi, dtype=float)
    nrm = np.sqrt(np.sum(g * g, axis=-1, keepdims=True))
    out = np.zeros_like(g)
    nz = has_normal(nrm[..., 0], h)
    out[nz] = g[nz] / nrm[nz]
    return out


def delta(phi, grad_phi, eps):
    """Regularized Dirac delta |grad H(phi)| of Eq. (delta) (chain rule through d(phi))."""
    phi = np.asarray(phi, dtype=float)
    _, dH, _, _, zone = heaviside_parts(phi, eps)
    g = np.sqrt(np.sum(np.asarray(grad_phi, dtype=float) ** 2, axis=-1))
    out = np.zeros_like(phi)
    out[zone] = dH[zone] * ddist_dphi(phi[zone], eps) * g[zone]
    return out


def dilation_coefficient(rho_l, rho_g):
    """c_1 = 1/rho_g - 1/rho_l, the factor of mdot delta in div u.

    Reading of the sign: Eq. (evaporDil) prints mdot (1/rho_l - 1/rho_g) delta, but the paper's own 1D solution
    (App. A, Eq. stefan_diffuse_velocity: u = u_bar + mdot (1 - H)(1/rho_g - 1/rho_l) with the liquid where H = 1)
    has div u = mdot (1/rho_g - 1/rho_l) delta, the derivation of variant 1 (Sec. 2.3.2) names c_1 = 1/rho_g -
    1/rho_l with c_1 mdot delta = div u, and evaporation (mdot > 0, liquid turning into the lighter gas) expands the
    volume.  The printed bracket is taken as reversed: v > 0 for mdot > 0 and rho_g < rho_l."""
    return 1.0 / rho_g - 1.0 / rho_l


def dilation_rate(mdot, phi, grad_phi, eps, rho_l, rho_g):
    """Regularized evaporative dilation rate, Eq. (evaporDil) with the sign of App. A: mdot c_1 delta."""
    return np.asarray(mdot, dtype=float) * dilation_coefficient(rho_l, rho_g) * delta(phi, grad_phi, eps)


def corrected_strain(eps_tensor, n, active=True):
    """Corrected rate of deformation, Eq. (modified_rate_of_deformation): eps - tr(eps) n (x) n.

    eps_tensor[..., d, d], n[..., d]; ``active`` gates the correction (interface zone)."""
    e = np.asarray(eps_tensor, dtype=float)
    tr = np.trace(e, axis1=-2, axis2=-1)
    corr = tr[..., None, None] * n[..., :, None] * n[..., None, :]
    act = np.asarray(active, dtype=float)
    return e - act[..., None, None] * corr if act.ndim else e - act * corr
