"""One time step of the coupled problem (test infrastructure): the Navier-Stokes step and Algorithm 2.

Algorithm 1 of the paper alternates the level-set solver (Algorithm 2) and the Navier-Stokes solver; the step here
takes them in the order velocity first, then level set, each once:

  1. Navier-Stokes with Picard iterations (params newton = 0) or Newton's method (newton = 1, App. D: "consistently
     linearized ... full Newton"): the Picard operator K(u^(k)) is linearized about the latest iterate u^(k)
     (u^(0) = u^n) and gives the nonlinear residual R^(k) = [f; g] - K(u^(k)) [u^(k); p^(k)]; a Picard iteration solves
     K(u^(k)) [u^(k+1); p^(k+1)] = [f; g], a Newton iteration solves J(u^(k)) [du; dp] = R^(k) with the Jacobian J,
     the operator with the Newton term (x . grad) u^(k), and adds the correction.  At most `picard_iters` iterations,
     stopping before an iteration k >= 1 once |R^(k)| <= picard_atol (the table's 1e-10 for the Navier-Stokes
     nonlinear solver); with picard_iters = 1 the Picard step is semi-implicit. The time discretization is
     BDF1 (c_m = 1/dt, u* = u^n) or, given u^(n-1), BDF2 (c_m = 3/(2 dt), u* = (4 u^n - u^(n-1)) / 3); with A the
     momentum operator of oracle.momentum for u0 = u^(k), newton = 0 and that c_m (A u = rho c_m u + rho (u^(k) .
     grad) u + viscous(u)),
        [A, -B^T; B, 0] [u^(n+1); p^(n+1)] = [f; g],   f_(i,c) = sum_q W N_i rho (c_m u*_c + g_c),
     g the continuity right-hand side (oracle.saddle), Dirichlet rows of f equal to those of u^n: the velocity on
     the Dirichlet faces keeps its value (walls at rest where u^n is 0 there, an inflow where it is not; the data
     are lifted into the free rows, oracle.saddle.lifted_matrix).  With a surface
     tension coefficient alpha != 0, f also carries the surface-tension force of Eq. (surfaceTension)
     (oracle.surface) with the projected normal and the regularized curvature of phi^n (Algorithm 2 step 3 of the
     previous step).
  2. Level set, Algorithm 2: the advection fixed point (oracle.geometry.advect_levelset) with the velocity u^(n+1)
     and `fp_iters` passes; the advected field clamped to [-1, 1]; its projected normal (Eq.
     normal_vector_regularized); `reinit_steps` reinitialization steps with that normal frozen, starting from the
     clamped field.
Returns (phi^(n+1), u^(n+1), p^(n+1)).
"""
from __future__ import annotations

import numpy as np

from . import fe, geometry, momentum, saddle, surface


def mass_load(pb: momentum.Problem, u: np.ndarray, gvec=(0.0, 0.0, 0.0)) -> np.ndarray:
    """f_(i,c) = sum_q W N_i rho(phi) (c_m u_c + g_c): the assembled operator of a copy of the problem with no
    viscosity, no convection and no Newton term (so it is rho c_m M) applied to u, plus the body-force load."""
    prm = dict(pb.params)
    prm.update(mu_l=0.0, mu_g=0.0, newton=0)
    mp = momentum.Problem(mesh=pb.mesh, params=prm, phi=pb.phi, u0=np.zeros_like(pb.u0), mdot=pb.mdot,
                          rho_mode=pb.rho_mode)
    f = momentum.assemble(mp) @ u
    if any(gvec):
        f = f + saddle.body_force_load(pb, gvec)
    f[pb.constrained()] = 0.0
    return f


def time_step(mesh_u: fe.Mesh, params: dict, phi: np.ndarray, u: np.ndarray, p: np.ndarray, mdot: np.ndarray,
              fp_iters: int = 2, reinit_steps: int = 2, gvec=(0.0, 0.0, 0.0), u_prev=None, picard_iters: int = 1,
              picard_atol: float = 0.0, residuals=None, alpha: float = 0.0):
    prm = dict(params)
    newton = int(prm.get("newton", 1)) != 0
    prm["newton"] = 0  # the Picard operator: residuals, and the Picard iterations' solves
    prm["c_mass"] = (1.0 if u_prev is None else 1.5) / prm["dt"]
    ustar = np.array(u, dtype=float) if u_prev is None else (4.0 * np.asarray(u) - np.asarray(u_prev)) / 3.0
    pb = momentum.Problem(mesh=mesh_u, params=prm, phi=np.clip(phi, -1.0, 1.0), u0=np.array(u, dtype=float),
                          mdot=np.array(mdot, dtype=float))
    f = mass_load(pb, ustar, gvec)
    mesh1 = fe.Mesh(mesh_u.n * mesh_u.n_sub, 1, mesh_u.L)  # the level-set mesh
    if alpha != 0.0:
        n0 = geometry.projected_normal(mesh1, pb.phi, prm.get("eta_n", 2.0))
        kappa = geometry.curvature(mesh1, n0, prm.get("eta_kappa", 2.0))
        f = f + surface.surface_tension_rhs(pb, n0, kappa, alpha)
        f[pb.constrained()] = 0.0
    mask = pb.constrained()
    f[mask] = np.asarray(u, dtype=float)[mask]  # Dirichlet data: the boundary values of u^n
    u1, p1 = np.array(u, dtype=float), np.array(p, dtype=float)
    nu3 = 3 * mesh_u.n_u
    for it in range(picard_iters):
        pb.u0 = u1
        if it > 0 or newton:
            K, g = saddle.lifted_matrix(pb)
            rvec = np.concatenate([f, g]) - K @ np.concatenate([u1, p1])
            res = float(np.linalg.norm(rvec))
            if it > 0:
                if residuals is not None:
                    residuals.append(res)
                if res <= picard_atol:
                    break
        if newton:
            # Newton: the Jacobian of the residual is the operator with the (x . grad) u^(k) term (App. D); the
            # correction has zero Dirichlet data (u^(k) already carries the boundary values)
            pn = momentum.Problem(mesh=mesh_u, params=dict(prm, newton=1), phi=pb.phi, u0=u1, mdot=pb.mdot)
            du, dp = saddle.solve(pn, rvec[:nu3], g=rvec[nu3:])
            u1, p1 = u1 + du, p1 + dp
        else:
            u1, p1 = saddle.solve(pb, f)
    adv, _ = geometry.advect_levelset(mesh_u, np.clip(phi, -1.0, 1.0), u1, mdot, prm, fp_iters)
    adv = np.clip(adv, -1.0, 1.0)
    n = geometry.projected_normal(mesh1, adv, prm.get("eta_n", 2.0))
    psi, _ = geometry.reinitialize(mesh1, adv, n, prm["eps"], prm["dtau"], reinit_steps, psi0=adv)
    return psi, u1, p1
