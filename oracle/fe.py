"""Finite-element building blocks of the oracle (test infrastructure, see package docstring).

Discretization of Sec. 2.5: continuous Lagrange elements on hexahedra, velocity degree k_u = 2 (3 also supported),
level set / pressure space degree 1, integrals evaluated with (k + 1)^dim Gauss points.  Support points are the
Gauss-Lobatto points of the reference interval [0, 1] (for k = 1, 2 they are the equispaced points).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def gauss_lobatto_points(p: int) -> np.ndarray:
    if p == 1:
        return np.array([0.0, 1.0])
    if p == 2:
        return np.array([0.0, 0.5, 1.0])
    if p == 3:
        r = 1.0 / math.sqrt(5.0)
        return np.array([0.0, 0.5 * (1.0 - r), 0.5 * (1.0 + r), 1.0])
    raise ValueError(f"degree {p} not supported")


def gauss_rule(nq: int) -> tuple[np.ndarray, np.ndarray]:
    """Gauss-Legendre points and weights on [0, 1] (library routine, mapped from [-1, 1])."""
    t, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange_1d(nodes: np.ndarray, x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """V[a, q] = l_a(x_q) and D[a, q] = l_a'(x_q) for the Lagrange polynomials l_a of ``nodes`` (product formula)."""
    m = len(nodes)
    x = np.asarray(x, dtype=float)
    V = np.ones((m, x.size))
    D = np.zeros((m, x.size))
    for a in range(m):
        for b in range(m):
            if b != a:
                V[a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
        for k in range(m):
            if k == a:
                continue
            term = np.full(x.size, 1.0 / (nodes[a] - nodes[k]))
            for b in range(m):
                if b != a and b != k:
                    term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            D[a] += term
    return V, D


@dataclass
class TensorBasis:
    """3D basis of Q_p on one cell of size h evaluated at the tensor points x_q (reference coords ``pts``).

    N[i, q] = N_i(x_q); G[b, i, q] = d N_i / d x_b (physical); local node index i = a + (p+1)(b + (p+1)c)."""

    p: int
    N: np.ndarray
    G: np.ndarray


def tensor_basis(p: int, pts: np.ndarray, h: float) -> TensorBasis:
    V, D = lagrange_1d(gauss_lobatto_points(p), pts)
    m, nq = V.shape
    N = np.einsum("ax,by,cz->cbazyx", V, V, V).reshape(m ** 3, nq ** 3)
    Gx = np.einsum("ax,by,cz->cbazyx", D, V, V).reshape(m ** 3, nq ** 3) / h
    Gy = np.einsum("ax,by,cz->cbazyx", V, D, V).reshape(m ** 3, nq ** 3) / h
    Gz = np.einsum("ax,by,cz->cbazyx", V, V, D).reshape(m ** 3, nq ** 3) / h
    return TensorBasis(p=p, N=N, G=np.stack([Gx, Gy, Gz]))


def iso_q1_1d(x: np.ndarray, n_sub: int) -> tuple[np.ndarray, np.ndarray]:
    """V[a, q], D[a, q] (reference derivative) of the n_sub + 1 piecewise-linear hat functions of [0, 1] subdivided
    n_sub times (nodes a / n_sub) at the points x.  A point lies in the sub-interval floor(n_sub x), clamped to
    n_sub - 1: on an interior node it takes the upper sub-interval's slopes.  For n_sub = 1 these are the Q1 shape
    functions 1 - x, x."""
    x = np.asarray(x, dtype=float)
    V = np.zeros((n_sub + 1, x.size))
    D = np.zeros((n_sub + 1, x.size))
    k = np.clip(np.floor(n_sub * x).astype(int), 0, n_sub - 1)
    xi = n_sub * x - k
    for q in range(x.size):
        V[k[q], q] += 1.0 - xi[q]
        V[k[q] + 1, q] += xi[q]
        D[k[q], q] -= n_sub
        D[k[q] + 1, q] += n_sub
    return V, D


def levelset_basis(n_sub: int, pts: np.ndarray, h: float) -> TensorBasis:
    """Level-set shape functions on one velocity cell of size h at the tensor points (reference coords ``pts``): Q1
    on each of the n_sub^3 sub-cells of the cell (the level-set mesh subdivided n_sub times per direction, Sec. 2.5),
    (n_sub + 1)^3 local nodes, local index a + (n_sub + 1)(b + (n_sub + 1)c); n_sub = 1 is the Q1 basis."""
    V, D = iso_q1_1d(pts, n_sub)
    m, nq = V.shape
    N = np.einsum("ax,by,cz->cbazyx", V, V, V).reshape(m ** 3, nq ** 3)
    Gx = np.einsum("ax,by,cz->cbazyx", D, V, V).reshape(m ** 3, nq ** 3) / h
    Gy = np.einsum("ax,by,cz->cbazyx", V, D, V).reshape(m ** 3, nq ** 3) / h
    Gz = np.einsum("ax,by,cz->cbazyx", V, V, D).reshape(m ** 3, nq ** 3) / h
    return TensorBasis(p=1, N=N, G=np.stack([Gx, Gy, Gz]))


def tensor_weights(w1: np.ndarray, h: float) -> np.ndarray:
    """W_q = w_x w_y w_z h^3 for q = qx + nq (qy + nq qz)."""
    return np.einsum("x,y,z->zyx", w1, w1, w1).ravel() * h ** 3


def tensor_points(t1: np.ndarray) -> np.ndarray:
    """(nq^3, 3) reference coordinates of the tensor points, x fastest."""
    Z, Y, X = np.meshgrid(t1, t1, t1, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


@dataclass
class Mesh:
    """Uniform n^3 hex mesh of [0, L]^3 with Q_p velocity nodes, Q1 pressure nodes, and Q1 level-set nodes on the mesh
    subdivided n_sub times per direction (Sec. 2.5; n_sub = 1: the level set shares the pressure nodes)."""

    n: int
    p: int
    L: float
    n_sub: int = 1

    @property
    def h(self) -> float:
        return self.L / self.n

    @property
    def m(self) -> int:  # Q_p nodes per axis
        return self.p * self.n + 1

    @property
    def n_u(self) -> int:
        return self.m ** 3

    @property
    def n_phi(self) -> int:  # level-set (and mass-flux) nodes
        return (self.n_sub * self.n + 1) ** 3

    @property
    def n_p(self) -> int:  # pressure nodes (Q1 on the velocity mesh)
        return (self.n + 1) ** 3

    def cells(self) -> np.ndarray:
        """(n^3, 3) integer cell coordinates (cx, cy, cz), cell index cx + n (cy + n cz)."""
        r = np.arange(self.n)
        Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def dofs_u(self, cells: np.ndarray | None = None) -> np.ndarray:
        """(ncell, (p+1)^3) global Q_p node indices of each cell, local order a + (p+1)(b + (p+1)c)."""
        cells = self.cells() if cells is None else cells
        p, m = self.p, self.m
        r = np.arange(p + 1)
        C, B, A = np.meshgrid(r, r, r, indexing="ij")
        A, B, C = A.ravel(), B.ravel(), C.ravel()
        gx = p * cells[:, 0:1] + A[None]
        gy = p * cells[:, 1:2] + B[None]
        gz = p * cells[:, 2:3] + C[None]
        return gx + m * (gy + m * gz)

    def dofs_p(self, cells: np.ndarray | None = None) -> np.ndarray:
        """(ncell, 8) global Q1 pressure node indices of each cell."""
        cells = self.cells() if cells is None else cells
        m1 = self.n + 1
        r = np.arange(2)
        C, B, A = np.meshgrid(r, r, r, indexing="ij")
        A, B, C = A.ravel(), B.ravel(), C.ravel()
        return (cells[:, 0:1] + A[None]) + m1 * ((cells[:, 1:2] + B[None]) + m1 * (cells[:, 2:3] + C[None]))

    def dofs_phi(self, cells: np.ndarray | None = None) -> np.ndarray:
        """(ncell, (n_sub+1)^3) global level-set node indices of each cell (local order a + (n_sub+1)(b + ...));
        for n_sub = 1 the 8 Q1 nodes (the pressure nodes)."""
        cells = self.cells() if cells is None else cells
        k, ml = self.n_sub, self.n_sub * self.n + 1
        r = np.arange(k + 1)
        C, B, A = np.meshgrid(r, r, r, indexing="ij")
        A, B, C = A.ravel(), B.ravel(), C.ravel()
        return (k * cells[:, 0:1] + A[None]) + ml * ((k * cells[:, 1:2] + B[None]) + ml * (k * cells[:, 2:3] + C[None]))

    def dirichlet_nodes(self, faces: int) -> np.ndarray:
        """Boolean [n_u] mask of Q_p nodes on the selected faces; bit 2*axis is the face x_axis = 0, bit 2*axis+1
        the face x_axis = L."""
        m = self.m
        r = np.arange(m)
        Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
        idx = [X.ravel(), Y.ravel(), Z.ravel()]
        mask = np.zeros(m ** 3, dtype=bool)
        for ax in range(3):
            if faces & (1 << (2 * ax)):
                mask |= idx[ax] == 0
            if faces & (1 << (2 * ax + 1)):
                mask |= idx[ax] == m - 1
        return mask
