"""Level-set geometry sub-solver by assembled Gauss quadrature and direct sparse solves (test infrastructure).

Steps 1 to 3 of Algorithm 2 (level_set_solver) on the Q1 level-set space with 2^3 Gauss points (Sec. 2.5),
homogeneous Neumann conditions on every face (no constraint):

  advection           Eqs. (transport), (weakFormLevelSet), Crank-Nicolson in time, step 1 of Algorithm 2: a fixed
                      point phi^(k) -> u_Gamma(phi^(k)) (oracle.transport) -> phi^(k+1) solving
                      (M + theta dt C) phi^(k+1) = (M - (1 - theta) dt C) phi^n, C_ij = sum_q W N_i (u_Gamma . grad N_j).

  projected normal    Eq. (normal_vector_regularized): n - eta_n h^2 Laplace n = nbar, nbar the unit normal of
                      Eq. (normal_vector) at the point (zero where phi is flat, physics.has_normal).  Weak form per
                      component c:  (M + eta_n h^2 K) n_c = b_c,  b_(c,i) = sum_q W_q N_i nbar_c.
  curvature           Eqs. (curvature), (curvature_regularized): kappa - eta_k h^2 Laplace kappa = -div n_Gamma with
                      n_Gamma the Q1 projected normal:  (M + eta_k h^2 K) kappa = b,  b_i = -sum_q W_q N_i div n_h.
  reinitialization    Eq. (reinitialization), semi-implicit Euler in pseudo-time with the normal frozen:
                      (M / dtau + eps K_n) psi^(k+1) = M psi^k / dtau + (grad N_i . n, (1 - (psi^k)^2) / 2),
                      K_n,ij = sum_q W (grad N_i . n)(grad N_j . n); n at the point is the normalized Q1 projected
                      normal n_h / |n_h| (zero where |n_h| <= 1e-4), or the unit normal of the current phi.

h is the cell edge (the largest cell diagonal over sqrt(3) on a cube).  The filter constants default to
eta_n = eta_k = 2 (the paper's defaults).  The discrete solutions are computed by a sparse direct solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe, physics
from .levelset import _assemble, q1_rule
from .momentum import _chunks

NODAL_NORMAL_TINY = 1e-4  # |n_h| at a point at or below this: the frozen reinitialization normal is taken as 0


def helmholtz_matrix(mesh: fe.Mesh, c: float) -> sp.csr_matrix:
    """M + c K on Q1 (Neumann), c = eta h^2."""
    b1, W = q1_rule(mesh)
    Me = np.einsum("q,iq,jq->ij", W, b1.N, b1.N)
    Ke = np.einsum("q,biq,bjq->ij", W, b1.G, b1.G)
    Ae = Me + c * Ke
    return _assemble(mesh, lambda d1: np.broadcast_to(Ae, (d1.shape[0], 8, 8)))


def unit_normal_rhs(mesh: fe.Mesh, phi: np.ndarray) -> np.ndarray:
    """b[c, i] = sum_q W_q N_i nbar_c(x_q), nbar = grad phi_h / |grad phi_h| (Eq. normal_vector)."""
    b1, W = q1_rule(mesh)
    cells = mesh.cells()
    b = np.zeros((3, mesh.n_phi))
    for sl in _chunks(len(cells), 4096):
        d1 = mesh.dofs_phi(cells[sl])
        nq = physics.normal(np.einsum("nj,bjq->nqb", phi[d1], b1.G), mesh.h)   # [nc, nq, 3]
        for c in range(3):
            np.add.at(b[c], d1.ravel(), np.einsum("q,iq,nq->ni", W, b1.N, nq[..., c]).ravel())
    return b


def curvature_rhs(mesh: fe.Mesh, n_field: np.ndarray) -> np.ndarray:
    """b_i = -sum_q W_q N_i div n_h(x_q) for the Q1 vector field n_field [3, N_phi]."""
    b1, W = q1_rule(mesh)
    cells = mesh.cells()
    nf = np.asarray(n_field).reshape(3, -1)
    b = np.zeros(mesh.n_phi)
    for sl in _chunks(len(cells), 4096):
        d1 = mesh.dofs_phi(cells[sl])
        div = sum(np.einsum("nj,jq->nq", nf[c][d1], b1.G[c]) for c in range(3))      # [nc, nq]
        np.add.at(b, d1.ravel(), -np.einsum("q,iq,nq->ni", W, b1.N, div).ravel())
    return b


def projected_normal(mesh: fe.Mesh, phi: np.ndarray, eta_n: float = 2.0) -> np.ndarray:
    """[3, N_phi] Q1 projected normal (Eq. normal_vector_regularized)."""
    A = helmholtz_matrix(mesh, eta_n * mesh.h ** 2).tocsc()
    b = unit_normal_rhs(mesh, phi)
    lu = spla.splu(A)
    return np.stack([lu.solve(b[c]) for c in range(3)])


def curvature(mesh: fe.Mesh, n_field: np.ndarray, eta_k: float = 2.0) -> np.ndarray:
    """[N_phi] regularized curvature (Eq. curvature_regularized) of the Q1 normal field n_field."""
    A = helmholtz_matrix(mesh, eta_k * mesh.h ** 2).tocsc()
    return spla.spsolve(A, curvature_rhs(mesh, n_field))


def nodal_normal_at_qp(mesh: fe.Mesh, n_field: np.ndarray, d1: np.ndarray, b1) -> np.ndarray:
    """[nc, nq, 3] n_h(x_q) / |n_h(x_q)| (zero where |n_h| <= NODAL_NORMAL_TINY)."""
    nf = np.asarray(n_field).reshape(3, -1)
    v = np.stack([nf[c][d1] @ b1.N for c in range(3)], axis=-1)
    nrm = np.sqrt(np.sum(v * v, axis=-1, keepdims=True))
    out = np.zeros_like(v)
    ok = nrm[..., 0] > NODAL_NORMAL_TINY
    out[ok] = v[ok] / nrm[ok]
    return out


def _reinit_normal(mesh, phi, n_field, d1, b1):
    if n_field is None:
        return physics.normal(np.einsum("nj,bjq->nqb", phi[d1], b1.G), mesh.h)
    return nodal_normal_at_qp(mesh, n_field, d1, b1)


def reinit_matrix(mesh: fe.Mesh, phi, n_field, eps: float, dtau: float) -> sp.csr_matrix:
    """M / dtau + eps K_n with the frozen normal (nodal field n_field, or the unit normal of phi if None)."""
    b1, W = q1_rule(mesh)

    def elem(d1):
        n = _reinit_normal(mesh, phi, n_field, d1, b1)
        gn = np.einsum("biq,nqb->nqi", b1.G, n)
        M = np.einsum("q,iq,jq->ij", W, b1.N, b1.N)
        return M[None] / dtau + eps * np.einsum("q,nqi,nqj->nij", W, gn, gn)

    return _assemble(mesh, elem)


def reinit_rhs(mesh: fe.Mesh, phi, n_field, psi0: np.ndarray, dtau: float) -> np.ndarray:
    b1, W = q1_rule(mesh)
    cells = mesh.cells()
    r = np.zeros(mesh.n_phi)
    for sl in _chunks(len(cells), 4096):
        d1 = mesh.dofs_phi(cells[sl])
        n = _reinit_normal(mesh, phi, n_field, d1, b1)
        gn = np.einsum("biq,nqb->nqi", b1.G, n)
        psi = psi0[d1] @ b1.N
        re = np.einsum("q,iq,nq->ni", W, b1.N, psi) / dtau + np.einsum("q,nqi,nq->ni", W, gn, 0.5 * (1.0 - psi * psi))
        np.add.at(r, d1.ravel(), re.ravel())
    return r


def reinitialize(mesh: fe.Mesh, phi: np.ndarray, n_field, eps: float, dtau: float, steps: int, psi0=None):
    """psi^0 = phi (or psi0), then `steps` semi-implicit pseudo-time steps (Algorithm 2, step 2) with the normal
    frozen at tau = 0 (the nodal field n_field, or the unit normal of phi).  Returns (psi, |psi^steps -
    psi^(steps-1)|_2)."""
    A = reinit_matrix(mesh, phi, n_field, eps, dtau).tocsc()
    lu = spla.splu(A)
    psi = np.array(phi if psi0 is None else psi0, dtype=float)
    change = 0.0
    for _ in range(steps):
        new = lu.solve(reinit_rhs(mesh, phi, n_field, psi, dtau))
        change = float(np.linalg.norm(new - psi))
        psi = new
    return psi, change


def advection_step(mesh1: fe.Mesh, phi_n: np.ndarray, ug: np.ndarray, theta: float, dt: float) -> np.ndarray:
    """One Crank-Nicolson step of Eq. (weakFormLevelSet) with the nodal transport velocity ug [3, N_phi]:
    solves (M + theta dt C) phi = (M - (1 - theta) dt C) phi^n, C_ij = sum_q W N_i (u_Gamma . grad N_j)."""
    from . import levelset
    M = helmholtz_matrix(mesh1, 0.0)
    A = levelset.advection_matrix(mesh1, np.asarray(ug).ravel(), theta, dt)
    C = (A - M) / (theta * dt)
    rhs = M @ phi_n - (1.0 - theta) * dt * (C @ phi_n)
    return spla.spsolve(A.tocsc(), rhs)


def advect_levelset(mesh_u: fe.Mesh, phi_n: np.ndarray, u0: np.ndarray, mdot: np.ndarray, prm: dict,
                    fp_iters: int):
    """Step 1 of Algorithm 2: the fixed point between the transport velocity and the Crank-Nicolson advection
    (Eqs. transport, weakFormLevelSet):  phi^(0) = phi^n;  for k: u_Gamma^(k) = u_Gamma(u0, mdot, phi^(k)) (the variant
    of prm, closest-point projection of App. C for variants 2/3), then phi^(k+1) = advection_step(phi^n, u_Gamma^(k)).
    phi^(k) is clamped to [-1, 1] before the transport velocity (as the fields of set_fields are).  Returns
    (phi^(fp_iters), [|phi^(k+1) - phi^(k)|_2 for each k])."""
    from . import transport
    mesh1 = fe.Mesh(mesh_u.n * mesh_u.n_sub, 1, mesh_u.L)  # the level-set mesh
    phi_k = np.array(phi_n, dtype=float)
    changes = []
    for _ in range(fp_iters):
        ug, _ = transport.transport_velocity(mesh_u, np.clip(phi_k, -1.0, 1.0), u0, mdot, prm)
        new = advection_step(mesh1, phi_n, ug, prm["theta"], prm["dt"])
        changes.append(float(np.linalg.norm(new - phi_k)))
        phi_k = new
    return phi_k, changes
