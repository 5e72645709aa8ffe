"""Adjoint of the momentum apply (test infrastructure).

Loss  L(x, phi, mdot, u0) = w . A(phi, u0) x + w_p . (B x - g(phi, mdot))   (velocity block + divergence row of
Eq. weakNavierStokes, see oracle.momentum).  Gradients:
  g_x    = A^T w + B^T w_p                    (explicit transposes of the assembled matrices)
  g_u0, g_phi, g_mdot                         by the chain rule through the quadrature-point coefficients:
     dF_c/du0_b = rho d_b x_c,  dF_c/d(d_d u0_c) = [newton] rho x_d
     drho/dH = -rho^2 (1/rho_l - 1/rho_g)  (Eq. rhoEff),  dmu/dH = mu_l - mu_g  (Eq. muEff)
     dH/dphi = H'(d) d'(phi),  d delta/dphi = (H''(d) d'(phi)^2 + H'(d) d''(phi)) |grad phi|,
     d delta/d grad phi = H'(d) d'(phi) n,  dn/d grad phi = (I - n n^T)/|grad phi|           (Eqs. delta, normal_vector)
  the zone indicator is piecewise constant (zero derivative).
``loss`` evaluates L directly so that the gradients can be checked against central differences.
"""
from __future__ import annotations

import numpy as np

from . import momentum, physics


def loss(pb: momentum.Problem, x, w, w_p=None) -> float:
    y = momentum.assemble(pb) @ x
    val = float(w @ y)
    if w_p is not None:
        B, g = momentum.divergence(pb)
        val += float(w_p @ (B @ x - g))
    return val


def grad_x(pb: momentum.Problem, w, w_p=None):
    gx = momentum.assemble(pb).T @ w
    if w_p is not None:
        B, _ = momentum.divergence(pb)
        gx = gx + B.T @ w_p
    return gx


def param_gradients(pb: momentum.Problem, x, w, w_p=None):
    """(g_u0[3 N_u], g_phi[N_phi], g_mdot[N_phi]) by hand-coded quadrature-point derivatives."""
    mesh, prm = pb.mesh, pb.params
    Nu = mesh.n_u
    mask = pb.constrained()
    xt = np.where(mask, 0.0, x).reshape(3, -1)
    wt = np.where(mask, 0.0, w).reshape(3, -1)
    g_u0 = np.zeros((3, Nu))
    g_phi = np.zeros(mesh.n_phi)
    g_mdot = np.zeros(mesh.n_phi)
    cm = prm["c_mass"]
    newton = float(int(prm.get("newton", 1)))
    eps = prm["eps"]
    k_rho = 1.0 / prm["rho_l"] - 1.0 / prm["rho_g"]                 # d(1/rho)/dH, Eq. (rhoEff)
    k_dil = physics.dilation_coefficient(prm["rho_l"], prm["rho_g"])  # v = mdot k_dil delta, Eq. (evaporDil)
    cells = mesh.cells()
    for sl in momentum._chunks(len(cells)):
        q = momentum.qp_fields(pb, cells[sl])
        W, bu, b1, du, d1 = q["W"], q["bu"], q["b1"], q["du"], q["d1"]
        bl, dl = q["bl"], q["dl"]  # level-set space (phi, mdot); b1, d1: pressure space (w_p)
        X = np.einsum("nci,iq->nqc", np.stack([xt[c][du] for c in range(3)], 1), bu.N)
        G = np.einsum("nci,biq->nqcb", np.stack([xt[c][du] for c in range(3)], 1), bu.G)
        Om = np.einsum("nci,iq->nqc", np.stack([wt[c][du] for c in range(3)], 1), bu.N)
        OmG = np.einsum("nci,biq->nqcb", np.stack([wt[c][du] for c in range(3)], 1), bu.G)
        rho, mu, n, z, U, GU = q["rho"], q["mu"], q["n"], q["z"], q["U"], q["GU"]
        Wq = W[None, :]
        # d L / d u0 at the quadrature point
        dU = Wq[..., None] * rho[..., None] * np.einsum("nqc,nqcb->nqb", Om, G)
        dGU = newton * (Wq * rho)[..., None, None] * np.einsum("nqc,nqd->nqcd", Om, X)
        gu = np.einsum("iq,nqb->nbi", bu.N, dU) + np.einsum("diq,nqbd->nbi", bu.G, dGU)
        for c in range(3):
            np.add.at(g_u0[c], du.ravel(), gu[:, c, :].ravel())
        # coefficient sensitivities
        F_over_rho = (cm * X + np.einsum("nqb,nqcb->nqc", U, G) + newton * np.einsum("nqcd,nqd->nqc", GU, X))
        dL_drho = Wq * np.einsum("nqc,nqc->nq", Om, F_over_rho)
        eps_t = 0.5 * (G + np.swapaxes(G, -1, -2))
        tr = np.trace(G, axis1=-2, axis2=-1)
        eps_mod = eps_t - (z * tr)[..., None, None] * n[..., :, None] * n[..., None, :]
        dL_dmu = Wq * 2.0 * np.einsum("nqcb,nqcb->nq", OmG, eps_mod)
        dL_dn = -(Wq * 2.0 * mu * z * tr)[..., None] * np.einsum("nqab,nqb->nqa", OmG + np.swapaxes(OmG, -1, -2), n)
        phi_q, gphi = q["phi"], q["gphi"]
        H, dH, d2H, _, zone = physics.heaviside_parts(phi_q, eps)
        dd = np.where(zone, physics.ddist_dphi(np.where(zone, phi_q, 0.0), eps), 0.0)
        d2d = np.where(zone, physics.d2dist_dphi2(np.where(zone, phi_q, 0.0), eps), 0.0)
        gnorm = np.sqrt(np.sum(gphi * gphi, axis=-1))
        if pb.rho_mode == "arithmetic":
            drho_dH = np.full_like(rho, prm["rho_l"] - prm["rho_g"])
        else:
            drho_dH = -rho * rho * k_rho
        dmu_dH = prm["mu_l"] - prm["mu_g"]
        dL_dphi = (dL_drho * drho_dH + dL_dmu * dmu_dH) * dH * dd
        dL_dg = np.zeros_like(gphi)
        nz = physics.has_normal(gnorm, mesh.h)
        proj = dL_dn - np.einsum("nqa,nqa->nq", dL_dn, n)[..., None] * n
        dL_dg[nz] = proj[nz] / gnorm[nz][:, None]
        dL_dm = np.zeros_like(phi_q)
        if w_p is not None:
            wp_q = w_p[d1] @ b1.N
            dL_dv = -Wq * wp_q
            delta = np.where(zone, dH * dd * gnorm, 0.0)
            dL_dm = dL_dv * k_dil * delta
            mq = q["mdot"]
            dL_dphi = dL_dphi + dL_dv * mq * k_dil * (d2H * dd * dd + dH * d2d) * gnorm
            dL_dg = dL_dg + (dL_dv * mq * k_dil * dH * dd)[..., None] * n
        gp = np.einsum("jq,nq->nj", bl.N, dL_dphi) + np.einsum("bjq,nqb->nj", bl.G, dL_dg)
        np.add.at(g_phi, dl.ravel(), gp.ravel())
        np.add.at(g_mdot, dl.ravel(), np.einsum("jq,nq->nj", bl.N, dL_dm).ravel())
    return g_u0.ravel(), g_phi, g_mdot
