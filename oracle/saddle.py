"""Velocity-pressure (saddle-point) system of the linearized Navier-Stokes step (test infrastructure).

Eq. (weakNavierStokes) with the Q1 pressure of Sec. 2.5 (k_u = p, k_p = 1): the momentum row carries the pressure
term -(div v, p), the continuity row (q, div x) = (q, v_dil) with the dilation rate of Eq. (evaporDil).  For the
velocity increment x and the pressure p:

    K [x; p] = [A x - B^T p;  B x] = [f;  g],      g_j = sum_q W N1_j v_dil

with A the velocity block of oracle.momentum (Dirichlet rows replaced by the identity) and B the divergence matrix
of oracle.momentum.divergence (Dirichlet velocity columns removed, so -B^T p vanishes on the constrained rows).
Faces whose bit is not set in `dirichlet_faces` are open: the natural condition of the weak form (zero traction)
holds there, which also fixes the pressure level.  With every face Dirichlet the pressure is determined only up to a
constant and K is singular; the solves here require an open face.

Dirichlet data.  The solves take the entries of f on the constrained DoFs as the prescribed velocity there (walls at
rest: 0; an inflow: its value) and lift them: they solve the system K_D [x; p] = [f; g] of `lifted_matrix`, whose
constrained rows are identity rows and whose free rows keep the constrained columns of the unconstrained A and B,
so x_c = f_c and the free rows see A_fc f_c and B_c f_c.  For f_c = 0 (homogeneous data) this is the system K.

Also the consistent load of a body force, f_(i,c) = sum_q W N_i rho(phi) g_c (the rho g term of Eq. momentum_balance),
and the outflow sum_(top face) of x . n, evaluated by face quadrature of the Q_p field (independently of B).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe, momentum, physics


def saddle_matrix(pb: momentum.Problem):
    """K [3 N_u + N_phi, 3 N_u + N_phi] and g [N_phi]."""
    A = momentum.assemble(pb)
    B, g = momentum.divergence(pb)
    K = sp.bmat([[A, -B.T], [B, None]]).tocsr()
    return K, g


def lifted_matrix(pb: momentum.Problem):
    """K_D = [A_D, -B^T; B_full, 0] and g: A_D is the unconstrained velocity block with its constrained rows replaced
    by identity rows (constrained columns kept), B_full the divergence matrix with every velocity column, and B
    (constrained columns removed) in the pressure term, which therefore vanishes on the constrained rows."""
    mask = pb.constrained()
    A = momentum.assemble(pb, apply_dirichlet=False)
    free = sp.diags((~mask).astype(float))
    A_D = (free @ A + sp.diags(mask.astype(float))).tocsr()
    B, g = momentum.divergence(pb)
    B_full, _ = momentum.divergence(pb, remove_constrained=False)
    return sp.bmat([[A_D, -B.T], [B_full, None]]).tocsr(), g


def apply(pb: momentum.Problem, x: np.ndarray, p: np.ndarray):
    """(A x - B^T p, B x)."""
    A = momentum.assemble(pb)
    B, _ = momentum.divergence(pb)
    return A @ x - B.T @ p, B @ x


def continuity_rhs(pb: momentum.Problem) -> np.ndarray:
    return momentum.divergence(pb)[1]


def solve(pb: momentum.Problem, f: np.ndarray, g=None):
    """Direct solve of K_D [x; p] = [f; g] (`lifted_matrix`: x = f on the constrained DoFs, lifted into the free
    rows; g the continuity right-hand side of the fields unless given); returns (x, p).  Needs an open face (else K
    is singular)."""
    if int(pb.params.get("dirichlet_faces", 0x3F)) & 0x3F == 0x3F:
        raise ValueError("the saddle-point system needs at least one open face")
    K, g_fields = lifted_matrix(pb)
    g = g_fields if g is None else g
    nu3 = 3 * pb.mesh.n_u
    sol = spla.spsolve(K.tocsc(), np.concatenate([f, g]))
    return sol[:nu3], sol[nu3:]


def body_force_load(pb: momentum.Problem, gvec) -> np.ndarray:
    """f_(i,c) = sum_q W N_i rho(phi_h(x_q)) g_c with the reciprocal density at the point; Dirichlet entries 0."""
    mesh = pb.mesh
    cells = mesh.cells()
    f = np.zeros(3 * mesh.n_u)
    t, w = fe.gauss_rule(mesh.p + 1)
    W = fe.tensor_weights(w, mesh.h)
    bu = fe.tensor_basis(mesh.p, t, mesh.h)
    bl = fe.levelset_basis(mesh.n_sub, t, mesh.h)
    prm = pb.params
    for sl in momentum._chunks(len(cells)):
        c = cells[sl]
        du, dl = mesh.dofs_u(c), mesh.dofs_phi(c)
        phi_q = pb.phi[dl] @ bl.N
        H = physics.heaviside_parts(phi_q, prm["eps"])[0]
        rho = physics.density(H, prm["rho_l"], prm["rho_g"], pb.rho_mode)
        fi = np.einsum("q,iq,nq->ni", W, bu.N, rho)                  # [nc, nloc]
        for comp in range(3):
            np.add.at(f, comp * mesh.n_u + du.ravel(), gvec[comp] * fi.ravel())
    f[pb.constrained()] = 0.0
    return f


def top_outflow(mesh: fe.Mesh, x: np.ndarray) -> float:
    """Integral of x_z over the face z = L by the (p+1)^2 Gauss rule of the Q_p trace (the field is polynomial there,
    so this is exact)."""
    m = mesh.m
    xz = x.reshape(3, -1)[2].reshape(m, m, m)[m - 1]               # [y, x] nodal values on the top face
    t, w = fe.gauss_rule(mesh.p + 1)
    x1 = fe.gauss_lobatto_points(mesh.p)
    V = np.array([[_lagrange(x1, a, tq) for a in range(mesh.p + 1)] for tq in t])   # [q, a]
    total = 0.0
    for cy in range(mesh.n):
        for cx in range(mesh.n):
            blk = xz[cy * mesh.p: cy * mesh.p + mesh.p + 1, cx * mesh.p: cx * mesh.p + mesh.p + 1]
            vals = V @ blk @ V.T                                       # [qy, qx]
            total += float(w @ vals @ w) * mesh.h * mesh.h
    return total


def _lagrange(nodes, a, x):
    v = 1.0
    for k, xk in enumerate(nodes):
        if k != a:
            v *= (x - xk) / (nodes[a] - xk)
    return v
