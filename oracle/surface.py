"""Surface-tension force vector by Gauss quadrature (test infrastructure).

Continuum surface force of Eq. (surfaceTension), f_st = alpha kappa n_Gamma delta_rho(phi), with the density-scaled
delta delta_rho = delta(phi) rho(phi) c_rho, c_rho = (rho_g - rho_l) / (rho_l rho_g ln(rho_g / rho_l)) (same section;
delta of Eq. (delta), rho the reciprocal interpolation of Eq. (rhoEff)), as the right-hand side of the momentum
equation in the Q_p velocity test space with the (p+1)^3 Gauss rule:

    b_(i,c) = sum_q W_q N_i(x_q) alpha kappa_h(x_q) n_c(x_q) delta(x_q) rho(x_q) c_rho,

kappa_h the Q1 curvature field, n = n_h / |n_h| the normalized Q1 normal field at the point (zero where |n_h| <= 1e-4),
phi, grad phi, delta and rho from the Q1 level set at the point.  Entries of Dirichlet-constrained velocity DoFs are
zero (homogeneous data).
"""
from __future__ import annotations

import numpy as np

from . import fe, physics
from .momentum import Problem, _chunks, velocity_rule

NODAL_NORMAL_TINY = 1e-4


def c_rho(rho_l: float, rho_g: float) -> float:
    return (rho_g - rho_l) / (rho_l * rho_g * np.log(rho_g / rho_l))


def density_scaled_delta(phi, grad_phi, eps, rho_l, rho_g):
    """delta_rho(phi) = delta(phi) rho(phi) c_rho at points (arrays)."""
    H, _, _, _, _ = physics.heaviside_parts(phi, eps)
    rho = physics.density(H, rho_l, rho_g)
    return physics.delta(phi, grad_phi, eps) * rho * c_rho(rho_l, rho_g)


def surface_tension_rhs(pb: Problem, n_field: np.ndarray, kappa: np.ndarray, alpha: float) -> np.ndarray:
    """[3 N_u] right-hand side b (component-major)."""
    mesh, prm = pb.mesh, pb.params
    t, W = velocity_rule(mesh)
    bu = fe.tensor_basis(mesh.p, t, mesh.h)
    b1 = fe.levelset_basis(mesh.n_sub, t, mesh.h)  # kappa, n and phi live on the level-set space
    nf = np.asarray(n_field).reshape(3, -1)
    out = np.zeros((3, mesh.n_u))
    cells = mesh.cells()
    for sl in _chunks(len(cells)):
        du = mesh.dofs_u(cells[sl])
        d1 = mesh.dofs_phi(cells[sl])
        phi_q = pb.phi[d1] @ b1.N
        gphi = np.einsum("nj,bjq->nqb", pb.phi[d1], b1.G)
        dr = density_scaled_delta(phi_q, gphi, prm["eps"], prm["rho_l"], prm["rho_g"])
        k_q = kappa[d1] @ b1.N
        v = np.stack([nf[c][d1] @ b1.N for c in range(3)], axis=-1)
        nrm = np.sqrt(np.sum(v * v, axis=-1, keepdims=True))
        n_q = np.zeros_like(v)
        ok = nrm[..., 0] > NODAL_NORMAL_TINY
        n_q[ok] = v[ok] / nrm[ok]
        s = W[None, :] * alpha * k_q * dr                     # [nc, nq]
        for c in range(3):
            np.add.at(out[c], du.ravel(), np.einsum("iq,nq->ni", bu.N, s * n_q[..., c]).ravel())
    out = out.ravel()
    out[pb.constrained()] = 0.0
    return out
