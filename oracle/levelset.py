"""Level-set advection and reinitialization operators by assembled Gauss quadrature (test infrastructure).

All on the Q1 level-set space with 2^3 Gauss points (Sec. 2.5), homogeneous Neumann on every face (no constraint).

  ADVECT      Crank-Nicolson left-hand side of Eq. (weakFormLevelSet) / Eq. (transport):
                A_ij = sum_q W_q [ N_i N_j + theta dt N_i (u_Gamma . grad N_j) ],  u_Gamma the Q1 nodal field.
  REINIT      semi-implicit Euler step of Eq. (reinitialization) (diffusive flux implicit, normal frozen):
                R_ij = sum_q W_q [ N_i N_j / dtau + eps (grad N_i . n)(grad N_j . n) ],  n = grad phi/|grad phi|.
  REINIT_RHS  explicit part of the same step, for psi0 the applied vector:
                r_i  = sum_q W_q [ N_i psi0 / dtau + (grad N_i . n) (1 - psi0^2) / 2 ]
              (the compressive flux is integrated by parts; its boundary term is dropped, psi ~ +-1 on the boundary).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fe, physics
from .momentum import _chunks


def q1_rule(mesh: fe.Mesh):
    t, w = fe.gauss_rule(2)
    return fe.tensor_basis(1, t, mesh.h), fe.tensor_weights(w, mesh.h)


def _normal_at_qp(mesh, phi, d1, b1):
    phin = phi[d1]
    return physics.normal(np.einsum("nj,bjq->nqb", phin, b1.G), mesh.h)


def _assemble(mesh: fe.Mesh, elem_fn) -> sp.csr_matrix:
    cells = mesh.cells()
    rows, cols, vals = [], [], []
    for sl in _chunks(len(cells), 4096):
        d1 = mesh.dofs_phi(cells[sl])
        Ae = elem_fn(d1)
        rows.append(np.repeat(d1[:, :, None], 8, axis=2).ravel())
        cols.append(np.repeat(d1[:, None, :], 8, axis=1).ravel())
        vals.append(Ae.ravel())
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(mesh.n_phi, mesh.n_phi)).tocsr()


def advection_matrix(mesh: fe.Mesh, u_gamma: np.ndarray, theta: float, dt: float) -> sp.csr_matrix:
    b1, W = q1_rule(mesh)
    ug = u_gamma.reshape(3, -1)

    def elem(d1):
        uq = np.stack([ug[c][d1] @ b1.N for c in range(3)], axis=-1)       # [nc, nq, 3]
        conv = np.einsum("nqb,bjq->nqj", uq, b1.G)                          # u . grad N_j
        M = np.einsum("q,iq,jq->ij", W, b1.N, b1.N)
        return M[None] + theta * dt * np.einsum("q,iq,nqj->nij", W, b1.N, conv)

    return _assemble(mesh, elem)


def reinit_matrix(mesh: fe.Mesh, phi: np.ndarray, eps: float, dtau: float) -> sp.csr_matrix:
    b1, W = q1_rule(mesh)

    def elem(d1):
        n = _normal_at_qp(mesh, phi, d1, b1)                                # [nc, nq, 3]
        gn = np.einsum("biq,nqb->nqi", b1.G, n)                             # grad N_i . n
        M = np.einsum("q,iq,jq->ij", W, b1.N, b1.N)
        return M[None] / dtau + eps * np.einsum("q,nqi,nqj->nij", W, gn, gn)

    return _assemble(mesh, elem)


def reinit_rhs(mesh: fe.Mesh, phi: np.ndarray, psi0: np.ndarray, dtau: float) -> np.ndarray:
    b1, W = q1_rule(mesh)
    cells = mesh.cells()
    r = np.zeros(mesh.n_phi)
    for sl in _chunks(len(cells), 4096):
        d1 = mesh.dofs_phi(cells[sl])
        n = _normal_at_qp(mesh, phi, d1, b1)
        gn = np.einsum("biq,nqb->nqi", b1.G, n)
        psi = psi0[d1] @ b1.N                                               # [nc, nq]
        re = np.einsum("q,iq,nq->ni", W, b1.N, psi) / dtau + np.einsum("q,nqi,nq->ni", W, gn, 0.5 * (1.0 - psi * psi))
        np.add.at(r, d1.ravel(), re.ravel())
    return r


def apply(mesh: fe.Mesh, mode: str, x: np.ndarray, phi: np.ndarray, u_gamma: np.ndarray | None, prm: dict):
    if mode == "advect":
        return advection_matrix(mesh, u_gamma, prm["theta"], prm["dt"]) @ x
    if mode == "reinit":
        return reinit_matrix(mesh, phi, prm["eps"], prm["dtau"]) @ x
    if mode == "reinit_rhs":
        return reinit_rhs(mesh, phi, x, prm["dtau"])
    raise ValueError(mode)
