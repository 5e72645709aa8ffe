"""Level-set transport velocity, variants 1/2/3, with closest-point projection (test infrastructure).

Variant 1, Eq. (transport_vel_local_continuous):   u_G(x) = u(x) + mdot/rho(x) n(x)
Variant 2, Eq. (transport_vel_extension_liquid):   u_G(x) = u(x_l(x)) + mdot/rho_l n(x)
Variant 3, Eq. (transport_vel_extension_gas):      u_G(x) = u(x_g(x)) + mdot/rho_g n(x)
evaluated at every Q1 node x.  x_l / x_g is the closest point of x on the isocontour phi = tanh(3/2) /
phi = tanh(-3/2), i.e. d = +3 eps / -3 eps (Sec. 2.3.3), found by the fixed-point iteration of App. C:
normal steps y <- y - (d(y) - d*) n(y) followed by one tangential step per tangent t_j that removes the tangential
part of y - x, repeated until |y^{k+1} - y^k| falls below the tolerance.

Readings where App. C leaves details open (the same on the GPU):
  * band: variant 2 projects nodes with -tanh(3) < phi < tanh(3/2), variant 3 nodes with -tanh(3/2) < phi < tanh(3);
    all other nodes use y = x.
  * a normal step moves y along n(y) by (d(y) - d*) / |grad d(y)|, d = d(phi_h); App. C writes the step for a
    distance function (|grad d| = 1), which d(phi_h) is only approximately when h is comparable to eps, and the
    plain step then converges slowly or overshoots.
  * a projection is a sequence of normal steps, stopping once |d(y) - d*| <= tol h: at most 20 from the node, at
    most 6 for a trial point of the tangential step (it starts next to the isocontour).  The iteration
    starts with the projection of x.  Each outer iteration then takes the tangential step (t0 = v - (v.n) n
    normalised, t1 = n x t0, v = e_x unless |n_x| > 0.9, then e_y; it maps y to x + ((y - x).n(y)) n(y)) followed
    by a projection.  The full tangential step is a gradient step on |y - x|^2 along the isocontour that
    overshoots by the ratio of the distance to the curvature radius, so the step is read as backtracked: its length
    factor is halved (1, 1/2, ..., 1/32) until the projected point reached the isocontour and is strictly closer
    to x; if none is, the current point is final.  The iteration also stops when |y^{k+1} - y^k| <= tol (cell units)
    or when an accepted step shortens |y - x| by at most 1e-12 of it (|y - x| is quadratic in the tangential error,
    so this pins y to ~1e-6 cells; it ends the zigzag along creases of the piecewise-trilinear isocontour).
    A node is flagged as not converged when the first projection does not reach the isocontour (e.g. it does not
    exist inside a thin droplet) or after kmax outer iterations.
  * positions are handled in cell units s = y / h of the level-set mesh (the velocity mesh subdivided n_sub times,
    h = h_u / n_sub) and clamped to the domain [0, n]^3; point location takes cell = clamp(floor(s), 0, n - 1) per
    axis; phi and grad phi are the trilinear Q1 interpolant of that cell, u the Q_p interpolant of the velocity cell
    located the same way at s / n_sub; d(phi) uses phi clamped to |phi| <= 1 - 2^-40.
  * n(x) is the normalised gradient of the Q1 interpolant at the node (point-located as above), 0 where it is
    negligible (physics.has_normal).
"""
from __future__ import annotations

import math

import numpy as np

from . import fe, physics

PHI_CLAMP = 1.0 - 2.0 ** -40
BACKTRACK = 6  # tangential step lengths tried per outer iteration
TRIAL_STEPS = 6  # normal steps of the projection of a trial point (it starts next to the isocontour)
STALL = 1e-12  # an accepted step shortening |y - x| by less than this fraction ends the iteration


class PointEval:
    """Point evaluation of the Q1 level set (on the level-set mesh: the velocity mesh subdivided n_sub times) and of
    the Q_p velocity, at positions s in level-set cell units (s = x / h_ls, h_ls = h / n_sub)."""

    def __init__(self, mesh: fe.Mesh, phi: np.ndarray, u0: np.ndarray):
        self.mesh = mesh
        self.phi = phi
        self.u0 = u0.reshape(3, -1)
        self.nodes = fe.gauss_lobatto_points(mesh.p)
        self.n_cells = mesh.n * mesh.n_sub  # level-set cells per axis
        self.h = mesh.h / mesh.n_sub        # level-set cell size

    def locate(self, s, n=None):
        n = self.n_cells if n is None else n
        k = [min(max(int(math.floor(s[a])), 0), n - 1) for a in range(3)]
        xi = [s[a] - k[a] for a in range(3)]
        return k, xi

    def phi_grad(self, s):
        (kx, ky, kz), (x, y, z) = self.locate(s)
        m1 = self.n_cells + 1
        h = self.h
        val = 0.0
        g = [0.0, 0.0, 0.0]
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    f = self.phi[(kx + a) + m1 * ((ky + b) + m1 * (kz + c))]
                    wx, wy, wz = (x if a else 1 - x), (y if b else 1 - y), (z if c else 1 - z)
                    dx, dy, dz = (1.0 if a else -1.0), (1.0 if b else -1.0), (1.0 if c else -1.0)
                    val += wx * wy * wz * f
                    g[0] += dx * wy * wz * f / h
                    g[1] += wx * dy * wz * f / h
                    g[2] += wx * wy * dz * f / h
        return val, np.array(g)

    def velocity(self, s):
        (kx, ky, kz), xi = self.locate(np.asarray(s, dtype=float) / self.mesh.n_sub, self.mesh.n)
        p, m = self.mesh.p, self.mesh.m
        Vs = [fe.lagrange_1d(self.nodes, np.array([xi[a]]))[0][:, 0] for a in range(3)]
        out = np.zeros(3)
        for c in range(p + 1):
            for b in range(p + 1):
                for a in range(p + 1):
                    node = (p * kx + a) + m * ((p * ky + b) + m * (p * kz + c))
                    out += Vs[0][a] * Vs[1][b] * Vs[2][c] * self.u0[:, node]
        return out


def _unit(g):
    nrm = math.sqrt(float(g @ g))
    return (g / nrm if nrm > 0.0 else np.zeros(3)), nrm


def project(ev: PointEval, y: np.ndarray, d_target: float, eps: float, tol: float, max_steps: int = 20):
    """Normal steps y <- y - (d(y) - d*) / |grad d(y)| n(y) (App. C), in cell units, clamped to the domain.

    Returns (y, reached) with reached = |d(y) - d*| <= tol h at the returned point (h, cell units: the level-set
    mesh's)."""
    n = ev.n_cells
    h = ev.h
    y = y.copy()
    for _ in range(max_steps):
        ph, g = ev.phi_grad(y)
        ph = min(max(ph, -PHI_CLAMP), PHI_CLAMP)
        r = float(physics.distance(ph, eps)) - d_target
        if abs(r) <= tol * h:
            return y, True
        nv, nrm = _unit(g)
        if nrm == 0.0:
            return y, False
        grad_d = float(physics.ddist_dphi(ph, eps)) * nrm          # |grad d(phi_h)| at y
        y = np.clip(y - (r / grad_d / h) * nv, 0.0, float(n))
    ph, _ = ev.phi_grad(y)
    ph = min(max(ph, -PHI_CLAMP), PHI_CLAMP)
    return y, abs(float(physics.distance(ph, eps)) - d_target) <= tol * h


def tangential_part(ev: PointEval, sx: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Components of y - x along the tangents t0, t1 of the isocontour at y (App. C); zero if grad phi vanishes."""
    _, g = ev.phi_grad(y)
    nv, nrm = _unit(g)
    if nrm == 0.0:
        return np.zeros(3)
    v = np.array([0.0, 1.0, 0.0]) if abs(nv[0]) > 0.9 else np.array([1.0, 0.0, 0.0])
    t0, _ = _unit(v - float(v @ nv) * nv)
    t1 = np.cross(nv, t0)
    dlt = y - sx
    return float(dlt @ t0) * t0 + float(dlt @ t1) * t1


def closest_point(ev: PointEval, sx: np.ndarray, d_target: float, eps: float, tol: float, kmax: int):
    """Closest point (cell units) of node position sx on the isocontour d(phi) = d_target; returns (y, converged)."""
    n = float(ev.n_cells)
    y, on = project(ev, sx.astype(float), d_target, eps, tol)
    if not on:
        return y, False
    dist = math.sqrt(float((y - sx) @ (y - sx)))
    for _ in range(kmax):
        tp = tangential_part(ev, sx, y)
        accepted = False
        omega = 1.0
        for _ in range(BACKTRACK):
            y_new, on_new = project(ev, np.clip(y - omega * tp, 0.0, n), d_target, eps, tol, TRIAL_STEPS)
            dist_new = math.sqrt(float((y_new - sx) @ (y_new - sx)))
            if on_new and dist_new < dist:
                accepted = True
                break
            omega *= 0.5
        if not accepted:
            return y, True
        step = math.sqrt(float((y_new - y) @ (y_new - y)))
        gain = dist - dist_new
        y, dist = y_new, dist_new
        if step <= tol or gain <= STALL * dist:
            return y, True
    return y, False


def transport_velocity(mesh: fe.Mesh, phi: np.ndarray, u0: np.ndarray, mdot: np.ndarray, prm: dict,
                       nodes: np.ndarray | None = None, return_points: bool = False):
    """u_Gamma[3, len(nodes)] and the non-converged flag per node (all Q1 nodes if ``nodes`` is None); with
    return_points also the point y[3, len(nodes)] (cell units) whose velocity was taken (the closest point for the
    band nodes of variants 2/3, else the node)."""
    ev = PointEval(mesh, phi, u0)
    m1 = ev.n_cells + 1  # level-set nodes per axis
    nodes = np.arange(mesh.n_phi) if nodes is None else np.asarray(nodes)
    variant = int(prm.get("variant", 2))
    eps = prm["eps"]
    tol, kmax = prm.get("cpp_tol", 1e-10), int(prm.get("cpp_kmax", 50))
    ug = np.zeros((3, len(nodes)))
    flags = np.zeros(len(nodes), dtype=np.int32)
    pts = np.zeros((3, len(nodes)))
    u0v = u0.reshape(3, -1)
    for t, node in enumerate(nodes):
        i, j, k = node % m1, (node // m1) % m1, node // (m1 * m1)
        sx = np.array([i, j, k], dtype=float)
        phx = float(phi[node])
        _, g = ev.phi_grad(sx)
        nx = physics.normal(g, ev.h)
        mx = float(mdot[node])
        if variant == 1:
            H = physics.heaviside(np.array([phx]), eps)[0]
            rho = physics.density(H, prm["rho_l"], prm["rho_g"])
            if mesh.n_sub == 1:  # the node is a velocity node
                vnode = (mesh.p * i) + mesh.m * ((mesh.p * j) + mesh.m * (mesh.p * k))
                uval = u0v[:, vnode]
            else:
                uval = ev.velocity(sx)
            ug[:, t] = uval + mx / rho * nx
            pts[:, t] = sx
            continue
        if variant == 2:
            band = (-physics.PHI_GAS_BAND < phx) and (phx < physics.PHI_BAND)
            d_t, rho_t = 3.0 * eps, prm["rho_l"]
        else:
            band = (-physics.PHI_BAND < phx) and (phx < physics.PHI_GAS_BAND)
            d_t, rho_t = -3.0 * eps, prm["rho_g"]
        y = sx
        if band:
            y, ok = closest_point(ev, sx, d_t, eps, tol, kmax)
            flags[t] = 0 if ok else 1
        ug[:, t] = ev.velocity(y) + mx / rho_t * nx
        pts[:, t] = y
    if return_points:
        return ug, flags, pts
    return ug, flags
