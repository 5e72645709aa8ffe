"""Linearized momentum operator and divergence row by assembled full Gauss quadrature (test infrastructure).

Weak form of the Navier-Stokes equations, Eq. (weakNavierStokes) in App. D, linearized by Newton's method about
the velocity u0 (App. D: BDF2 + full Newton), for a velocity increment x with test function v:

  a(v, x) = sum_q W_q [ v_c F_c + d_b v_c T_cb ]
  F_c  = rho ( c_m x_c + (u0 . grad) x_c + [newton] (x . grad) u0_c )                       (inertia, convection)
  T_cb = 2 mu eps_mod(x)_cb,  eps = sym grad x,  eps_mod = eps - z tr(eps) n (x) n           Eqs. (stokesLaw),
                                                                                 (modified_rate_of_deformation)
  with rho, mu, n evaluated from phi_h at the quadrature point (Eqs. rhoEff, muEff, normal_vector) and z = 1 in
  the interface zone 0 < H < 1 for the corrected Stokes law (z = 0 for the standard one).

  Divergence row (continuity, Eq. continuity / first line of Eq. weakNavierStokes), Q1 test functions N^p_j:
    y_p[j] = sum_q W_q N^p_j (div x - v_dil),   v_dil from Eq. (evaporDil).

The quadrature-point coefficient is written as a 12 x 12 flux Jacobian C_q acting on [x_c, d_b x_c] so that the
element matrix is literally sum_q B_q^T (W_q C_q) B_q.  Homogeneous Dirichlet rows/columns on the selected faces
are replaced by the identity (the increment vanishes there, the applied vector is passed through).
Quadrature: (p+1)^3 Gauss points for both the velocity block and the divergence row (Sec. 2.5).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fe, physics


@dataclass
class Problem:
    """Mesh + parameters + coefficient fields of one operator instance."""

    mesh: fe.Mesh
    params: dict
    phi: np.ndarray      # [N_phi] Q1 nodal level set
    u0: np.ndarray       # [3 N_u] Q_p nodal linearization velocity
    mdot: np.ndarray     # [N_phi] Q1 nodal evaporative mass flux
    rho_mode: str = "reciprocal"

    @classmethod
    def from_workload(cls, wl, **over) -> "Problem":
        prm = dict(wl.params)
        prm.update(over)
        return cls(mesh=fe.Mesh(wl.n, wl.p, wl.L, int(prm.get("n_sub", 1))), params=prm,
                   phi=np.array(wl.phi, dtype=float),
                   u0=np.array(wl.u0, dtype=float), mdot=np.array(wl.mdot, dtype=float))

    def constrained(self) -> np.ndarray:
        """Boolean [3 N_u] mask of Dirichlet-constrained velocity DoFs."""
        node = self.mesh.dirichlet_nodes(int(self.params.get("dirichlet_faces", 0x3F)))
        return np.tile(node, 3)


def velocity_rule(mesh: fe.Mesh):
    t, w = fe.gauss_rule(mesh.p + 1)
    return t, fe.tensor_weights(w, mesh.h)


def qp_fields(pb: Problem, cells: np.ndarray):
    """Coefficient fields at the velocity quadrature points of ``cells`` (arrays [ncell, nq, ...]).

    phi and mdot are interpolated from the level-set space (bl, dl: Q1 on the cell's n_sub^3 sub-cells, Sec. 2.5);
    b1, d1 are the Q1 pressure-space shape functions and nodes (the divergence row's test functions)."""
    mesh, prm = pb.mesh, pb.params
    t, W = velocity_rule(mesh)
    bu = fe.tensor_basis(mesh.p, t, mesh.h)
    b1 = fe.tensor_basis(1, t, mesh.h)
    bl = fe.levelset_basis(mesh.n_sub, t, mesh.h)
    du = mesh.dofs_u(cells)
    d1 = mesh.dofs_p(cells)
    dl = mesh.dofs_phi(cells)
    phin = pb.phi[dl]                                          # [nc, (n_sub+1)^3]
    phi_q = phin @ bl.N                                        # [nc, nq]
    gphi = np.einsum("nj,bjq->nqb", phin, bl.G)               # [nc, nq, 3]
    mdot_q = pb.mdot[dl] @ bl.N
    u0 = pb.u0.reshape(3, -1)
    un = np.stack([u0[c][du] for c in range(3)], axis=1)      # [nc, 3, nloc]
    U = np.einsum("nci,iq->nqc", un, bu.N)                     # [nc, nq, 3]
    GU = np.einsum("nci,biq->nqcb", un, bu.G)                  # [nc, nq, 3, 3]  GU[c, b] = d_b u0_c
    H, _, _, _, zone = physics.heaviside_parts(phi_q, prm["eps"])
    rho = physics.density(H, prm["rho_l"], prm["rho_g"], pb.rho_mode)
    mu = physics.viscosity(H, prm["mu_l"], prm["mu_g"])
    n = physics.normal(gphi, mesh.h)
    vdil = physics.dilation_rate(mdot_q, phi_q, gphi, prm["eps"], prm["rho_l"], prm["rho_g"])
    if int(prm.get("stress", 1)) == 0:
        z = np.zeros_like(phi_q)
    elif int(prm.get("corr_zone", 0)) == 1:
        z = np.ones_like(phi_q)
    else:
        z = zone.astype(float)
    return dict(W=W, bu=bu, b1=b1, bl=bl, du=du, d1=d1, dl=dl, phi=phi_q, gphi=gphi, mdot=mdot_q, U=U, GU=GU, H=H,
                rho=rho, mu=mu, n=n, z=z, vdil=vdil, zone=zone)


def flux_jacobian(q: dict, prm: dict) -> np.ndarray:
    """C[nc, nq, 12, 12]: [F_c, T_cb] = C [x_d, d_e x_d]; index 0..2 values, 3 + 3 c + b gradients."""
    nc, nq = q["rho"].shape
    C = np.zeros((nc, nq, 12, 12))
    rho, mu, n, z = q["rho"], q["mu"], q["n"], q["z"]
    cm = prm["c_mass"]
    newton = float(int(prm.get("newton", 1)))
    I3 = np.eye(3)
    for c in range(3):
        for d in range(3):
            C[:, :, c, d] = rho * (cm * I3[c, d] + newton * q["GU"][:, :, c, d])
            for e in range(3):
                C[:, :, c, 3 + 3 * d + e] = rho * q["U"][:, :, e] * I3[c, d]
    for c in range(3):
        for b in range(3):
            for d in range(3):
                for e in range(3):
                    sym = 0.5 * (I3[c, d] * I3[b, e] + I3[b, d] * I3[c, e])
                    corr = z * I3[d, e] * n[:, :, c] * n[:, :, b]
                    C[:, :, 3 + 3 * c + b, 3 + 3 * d + e] = 2.0 * mu * (sym - corr)
    return C


def value_gradient_operator(bu: fe.TensorBasis) -> np.ndarray:
    """Bop[q, k, c, i]: maps element DoFs x[c, i] to [x_c, d_b x_c] at quadrature point q."""
    nloc, nq = bu.N.shape
    B = np.zeros((nq, 12, 3, nloc))
    for c in range(3):
        B[:, c, c, :] = bu.N.T
        for b in range(3):
            B[:, 3 + 3 * c + b, c, :] = bu.G[b].T
    return B


def element_matrices(pb: Problem, cells: np.ndarray) -> np.ndarray:
    """A_e[nc, 3*nloc, 3*nloc] with local DoF index c*nloc + i."""
    q = qp_fields(pb, cells)
    C = flux_jacobian(q, pb.params) * q["W"][None, :, None, None]
    B = value_gradient_operator(q["bu"])
    nq, _, _, nloc = B.shape
    Bf = B.reshape(nq, 12, 3 * nloc)
    T = np.matmul(C, Bf[None])                                       # (W_q C_q) B_q        [nc, nq, 12, 3 nloc]
    Bt = Bf.reshape(nq * 12, 3 * nloc).T                             # stacked B_q^T
    return np.matmul(Bt[None], T.reshape(len(T), nq * 12, 3 * nloc))  # sum_q B_q^T (W_q C_q) B_q


def _chunks(ncell: int, size: int = 512):
    for s in range(0, ncell, size):
        yield slice(s, min(ncell, s + size))


def assemble(pb: Problem, apply_dirichlet: bool = True) -> sp.csr_matrix:
    """Global velocity-block matrix [3 N_u, 3 N_u] (component-major DoFs c*N_u + node)."""
    mesh = pb.mesh
    cells = mesh.cells()
    Nu = mesh.n_u
    rows, cols, vals = [], [], []
    for sl in _chunks(len(cells)):
        Ae = element_matrices(pb, cells[sl])
        du = mesh.dofs_u(cells[sl])
        nloc = du.shape[1]
        g = (np.arange(3)[None, :, None] * Nu + du[:, None, :]).reshape(len(du), 3 * nloc)
        rows.append(np.repeat(g[:, :, None], 3 * nloc, axis=2).ravel())
        cols.append(np.repeat(g[:, None, :], 3 * nloc, axis=1).ravel())
        vals.append(Ae.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(3 * Nu, 3 * Nu)).tocsr()
    if apply_dirichlet:
        A = constrain(A, pb.constrained())
    return A


def constrain(A: sp.csr_matrix, mask: np.ndarray) -> sp.csr_matrix:
    """Zero constrained rows and columns and put 1 on their diagonal."""
    keep = sp.diags((~mask).astype(float))
    return (keep @ A @ keep + sp.diags(mask.astype(float))).tocsr()


def divergence(pb: Problem, remove_constrained: bool = True) -> tuple[sp.csr_matrix, np.ndarray]:
    """B[N_phi, 3 N_u] (constrained velocity columns removed unless remove_constrained is False) and source g[N_phi]
    of the divergence row."""
    mesh = pb.mesh
    cells = mesh.cells()
    Nu = mesh.n_u
    rows, cols, vals = [], [], []
    g = np.zeros(mesh.n_p)
    for sl in _chunks(len(cells)):
        q = qp_fields(pb, cells[sl])
        W, bu, b1 = q["W"], q["bu"], q["b1"]
        Be = np.einsum("q,jq,diq->jdi", W, b1.N, bu.G)                 # [8, 3, nloc]  (same for every cell)
        du, d1 = q["du"], q["d1"]
        nc, nloc = du.shape
        gcol = (np.arange(3)[None, :, None] * Nu + du[:, None, :])      # [nc, 3, nloc]
        rows.append(np.broadcast_to(d1[:, :, None, None], (nc, 8, 3, nloc)).ravel())
        cols.append(np.broadcast_to(gcol[:, None, :, :], (nc, 8, 3, nloc)).ravel())
        vals.append(np.broadcast_to(Be[None], (nc, 8, 3, nloc)).ravel())
        np.add.at(g, d1.ravel(), np.einsum("q,jq,nq->nj", W, b1.N, q["vdil"]).ravel())
    B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.n_p, 3 * Nu)).tocsr()
    if not remove_constrained:
        return B, g
    keep = sp.diags((~pb.constrained()).astype(float))
    return (B @ keep).tocsr(), g


def apply(pb: Problem, x: np.ndarray, with_divergence: bool = False):
    """y = A x (and y_p = B x - g)."""
    y = assemble(pb) @ x
    if not with_divergence:
        return y
    B, g = divergence(pb)
    return y, B @ x - g


def cells_touching_nodes(mesh: fe.Mesh, nodes: np.ndarray, degree: int) -> np.ndarray:
    """Unique cells whose closure contains the given nodes of the degree-``degree`` lattice."""
    m = degree * mesh.n + 1
    gi = np.stack([nodes % m, (nodes // m) % m, nodes // (m * m)], axis=1)
    out = set()
    for g in gi:
        opts = []
        for a in range(3):
            k, r = divmod(int(g[a]), degree)
            cand = [k - 1, k] if r == 0 else [k]
            opts.append([c for c in cand if 0 <= c < mesh.n])
        for cx in opts[0]:
            for cy in opts[1]:
                for cz in opts[2]:
                    out.add((cx, cy, cz))
    return np.array(sorted(out, key=lambda c: (c[2], c[1], c[0])), dtype=int).reshape(-1, 3)


def apply_rows(pb: Problem, x: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """Rows of y = A x for all 3 components of the given Q_p nodes, from the cells around them only.

    Returns y_rows[3, len(nodes)]."""
    mesh = pb.mesh
    Nu = mesh.n_u
    mask = pb.constrained()
    xt = np.where(mask, 0.0, x)
    cells = cells_touching_nodes(mesh, nodes, mesh.p)
    y = np.zeros(3 * Nu)
    for sl in _chunks(len(cells)):
        Ae = element_matrices(pb, cells[sl])
        du = mesh.dofs_u(cells[sl])
        nloc = du.shape[1]
        g = (np.arange(3)[None, :, None] * Nu + du[:, None, :]).reshape(len(du), 3 * nloc)
        ye = np.einsum("nij,nj->ni", Ae, xt[g])
        np.add.at(y, g.ravel(), ye.ravel())
    y = np.where(mask, x, y)
    return np.stack([y[c * Nu + nodes] for c in range(3)])


def divergence_rows(pb: Problem, x: np.ndarray, q1nodes: np.ndarray) -> np.ndarray:
    """Rows y_p[j] = (B x - g)[j] of the given Q1 pressure nodes, from the cells around them only."""
    mesh = pb.mesh
    Nu = mesh.n_u
    xt = np.where(pb.constrained(), 0.0, x)
    cells = cells_touching_nodes(mesh, q1nodes, 1)
    yp = np.zeros(mesh.n_p)
    for sl in _chunks(len(cells)):
        q = qp_fields(pb, cells[sl])
        W, bu, b1, du, d1 = q["W"], q["bu"], q["b1"], q["du"], q["d1"]
        xe = np.stack([xt[c * Nu + du] for c in range(3)], axis=1)               # [nc, 3, nloc]
        div = np.einsum("nci,ciq->nq", xe, bu.G)                                  # sum_c d_c x_c
        re = np.einsum("q,jq,nq->nj", W, b1.N, div - q["vdil"])
        np.add.at(yp, d1.ravel(), re.ravel())
    return yp[q1nodes]
