"""One time step of the coupled problem (test infrastructure): the Navier-Stokes step and Algorithm 2.

Algorithm 1 of the paper alternates the level-set solver (Algorithm 2) and the Navier-Stokes solver; the step here
takes them in the order velocity first, then level set, each once:

  1. Navier-Stokes, BDF1 with one Picard linearization about u^n (Eq. weakNavierStokes; App. D uses BDF2 and full
     Newton, see the module readings): with A the momentum operator of oracle.momentum for u0 = u^n, newton = 0 and
     c_m = 1/dt (so A u = rho u / dt + rho (u^n . grad) u + viscous(u)),
        [A, -B^T; B, 0] [u^(n+1); p^(n+1)] = [f; g],   f_(i,c) = sum_q W N_i rho (u^n_c / dt + g_c),
     g the continuity right-hand side (oracle.saddle), Dirichlet rows of f zero (walls at rest).
  2. Level set, Algorithm 2: the advection fixed point (oracle.geometry.advect_levelset) with the velocity u^(n+1)
     and `fp_iters` passes; the advected field clamped to [-1, 1]; its projected normal (Eq.
     normal_vector_regularized); `reinit_steps` reinitialization steps with that normal frozen, starting from the
     clamped field.
Returns (phi^(n+1), u^(n+1), p^(n+1)).
"""
from __future__ import annotations

import numpy as np

from . import fe, geometry, momentum, saddle


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
              fp_iters: int = 2, reinit_steps: int = 2, gvec=(0.0, 0.0, 0.0)):
    prm = dict(params)
    if int(prm.get("newton", 1)) != 0 or abs(prm["c_mass"] * prm["dt"] - 1.0) > 1e-12:
        raise ValueError("the step is BDF1 with a Picard linearization: newton = 0 and c_mass = 1/dt")
    pb = momentum.Problem(mesh=mesh_u, params=prm, phi=np.clip(phi, -1.0, 1.0), u0=np.array(u, dtype=float),
                          mdot=np.array(mdot, dtype=float))
    f = mass_load(pb, u, gvec)
    u1, p1 = saddle.solve(pb, f)
    mesh1 = fe.Mesh(mesh_u.n, 1, mesh_u.L)
    adv, _ = geometry.advect_levelset(mesh_u, np.clip(phi, -1.0, 1.0), u1, mdot, prm, fp_iters)
    adv = np.clip(adv, -1.0, 1.0)
    n = geometry.projected_normal(mesh1, adv, prm.get("eta_n", 2.0))
    psi, _ = geometry.reinitialize(mesh1, adv, n, prm["eps"], prm["dtau"], reinit_steps, psi0=adv)
    return psi, u1, p1
