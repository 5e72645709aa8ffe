"""Seeded synthetic inputs for the evaporation operators (shared by the oracle tests, the GPU tests and the bench).

This module holds no arithmetic of the method itself: it only builds node coordinates of the uniform hex mesh and
draws the nodal fields (level set, velocity, mass flux, applied vectors) that both the CPU oracle and the CUDA path
take as inputs.  The level set is the regularized indicator of Eq. (initial_phi), phi = tanh(d / (2 eps)), of a
signed distance d that is positive in the liquid (Sec. 2.2.2: phi > 0 liquid, phi < 0 gas).

Layouts (identical on both sides):
  * Q_p velocity nodes: (p*n+1)^3 points per component, lexicographic index i + M*(j + M*k), i fastest, M = p*n+1;
    the 1D node positions inside a cell are the Gauss-Lobatto points of degree p.
  * Vector fields are component-major: v[c*N + idx].
  * Q1 nodes (level set, mass flux, pressure space): (n+1)^3, same lexicographic order; with params "n_sub" = 2 the
    level set and the mass flux live on the Q1 nodes of the mesh subdivided twice per direction, (2n+1)^3 of them
    (the pressure stays on the (n+1)^3 nodes).

Workload recipes (domain [0, L]^3, L = 1, eps = one cell width h unless stated):
  * sphere:   d = R - |x - c|, R = 0.25, c = (0.5, 0.5, 0.5)                   (droplet, Sec. 3.2)
  * spheres:  d = max_k (R_k - |x - c_k|), 4 spheres, c_k ~ U[0.2, 0.8]^3, R_k ~ U[0.08, 0.2]
  * slab:     d = 0.5 - z (liquid below z = 0.5)                                (1D phase change, Sec. 3.1)
  * deformed: d = R(theta, varphi) - |x - c|, R = 0.3 (1 + 0.1 s), s a real spherical-harmonic sum up to l = 6
              with N(0,1) coefficients, normalised to max|s| = 1
  * velocity 'uniform': U[-1, 1] per DoF;  'fourier': sum over 1 <= |k|_inf <= 4 of a_k cos(2 pi k.x) +
    b_k sin(2 pi k.x), a_k, b_k ~ N(0, I_3), scaled to unit nodal RMS of |u|.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAUSS_LOBATTO = {
    1: np.array([0.0, 1.0]),
    2: np.array([0.0, 0.5, 1.0]),
    3: np.array([0.0, 0.5 - 0.5 / math.sqrt(5.0), 0.5 + 0.5 / math.sqrt(5.0), 1.0]),
}


def node_coords_1d(n: int, p: int, L: float = 1.0) -> np.ndarray:
    """1D coordinates of the Q_p nodes of an n-cell uniform line of length L (global index p*cell + a)."""
    h = L / n
    ref = GAUSS_LOBATTO[p]
    x = np.empty(p * n + 1)
    for c in range(n):
        x[p * c: p * c + p + 1] = (c + ref) * h
    x[-1] = L
    return x


def node_coords(n: int, p: int, L: float = 1.0) -> np.ndarray:
    """(N, 3) coordinates of the Q_p nodes in lexicographic order (x fastest)."""
    x = node_coords_1d(n, p, L)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def signed_distance(kind: str, pts: np.ndarray, rng: np.random.Generator | None = None, **kw) -> np.ndarray:
    if kind == "sphere":
        c = np.asarray(kw.get("center", (0.5, 0.5, 0.5)))
        R = kw.get("radius", 0.25)
        return R - np.linalg.norm(pts - c, axis=1)
    if kind == "spheres":
        k = kw.get("count", 4)
        centers = rng.uniform(0.2, 0.8, size=(k, 3))
        radii = rng.uniform(0.08, 0.2, size=k)
        d = np.full(pts.shape[0], -np.inf)
        for c, R in zip(centers, radii):
            d = np.maximum(d, R - np.linalg.norm(pts - c, axis=1))
        return d
    if kind == "slab":
        return kw.get("z0", 0.5) - pts[:, 2]
    if kind == "deformed":
        return _deformed_sphere_distance(pts, rng, lmax=kw.get("lmax", 6))
    raise ValueError(kind)


def _real_sph_harm_table(lmax: int, theta: np.ndarray, varphi: np.ndarray) -> list[np.ndarray]:
    """Real spherical harmonics (unnormalised associated-Legendre form) for 1 <= l <= lmax, all m."""
    from scipy.special import lpmv

    x = np.cos(theta)
    out = []
    for l in range(1, lmax + 1):
        for m in range(0, l + 1):
            P = lpmv(m, l, x)
            out.append(P * np.cos(m * varphi))
            if m > 0:
                out.append(P * np.sin(m * varphi))
    return out


def _deformed_sphere_distance(pts: np.ndarray, rng: np.random.Generator, lmax: int) -> np.ndarray:
    c = np.array([0.5, 0.5, 0.5])
    r = pts - c
    rad = np.linalg.norm(r, axis=1)
    theta = np.arccos(np.clip(r[:, 2] / np.maximum(rad, 1e-300), -1.0, 1.0))
    varphi = np.arctan2(r[:, 1], r[:, 0])
    basis = _real_sph_harm_table(lmax, theta, varphi)
    coef = rng.standard_normal(len(basis))
    # normalise on a fixed angular grid so max|s| = 1 independently of the mesh
    tg, pg = np.meshgrid(np.linspace(0, np.pi, 181), np.linspace(-np.pi, np.pi, 361), indexing="ij")
    sg = sum(a * b for a, b in zip(coef, _real_sph_harm_table(lmax, tg.ravel(), pg.ravel())))
    scale = 1.0 / np.max(np.abs(sg))
    s = scale * sum(a * b for a, b in zip(coef, basis))
    R = 0.3 * (1.0 + 0.1 * s)
    return R - rad


def fourier_velocity(n: int, p: int, rng: np.random.Generator, kmax: int = 4, L: float = 1.0) -> np.ndarray:
    """Random Fourier velocity at the Q_p nodes, component-major [3*N], unit nodal RMS of |u|.

    Evaluated separably: sum_k c_k exp(2 pi i k.x) factorises into 1D exponentials along x, y, z."""
    x = node_coords_1d(n, p, L)
    ks = np.arange(-kmax, kmax + 1)
    E = np.exp(2j * np.pi * np.outer(ks, x) / L)  # [k, node1d]
    K = len(ks)
    u = np.empty((3, len(x), len(x), len(x)))  # [c, z, y, x]
    kk = np.stack(np.meshgrid(ks, ks, ks, indexing="ij"), axis=0)  # [3, kz, ky, kx]
    mask = (np.max(np.abs(kk), axis=0) >= 1).astype(float)
    for c in range(3):
        a = rng.standard_normal((K, K, K))
        b = rng.standard_normal((K, K, K))
        coef = (a - 1j * b) * mask  # Re[(a - i b) e^{i t}] = a cos t + b sin t ; indices [kz, ky, kx]
        t = np.einsum("abc,cx->abx", coef, E)
        t = np.einsum("abx,by->ayx", t, E)
        t = np.einsum("ayx,az->zyx", t, E)
        u[c] = t.real
    u = u.reshape(3, -1)
    rms = math.sqrt(np.mean(np.sum(u * u, axis=0)))
    return (u / rms).ravel()


@dataclass
class Workload:
    """One synthetic problem: mesh size, degree, parameters and nodal fields (all float64, host)."""

    n: int
    p: int
    L: float
    params: dict
    phi: np.ndarray          # [N_phi]
    u0: np.ndarray           # [3*N_u]
    mdot: np.ndarray         # [N_phi]
    x: np.ndarray            # [3*N_u] applied velocity vector
    extra: dict = field(default_factory=dict)

    @property
    def n_u(self) -> int:
        return (self.p * self.n + 1) ** 3

    @property
    def n_phi(self) -> int:  # level-set nodes: Q1 on the mesh subdivided n_sub times (params "n_sub", default 1)
        return (int(self.params.get("n_sub", 1)) * self.n + 1) ** 3


def default_params(n: int, L: float = 1.0, ratio: float = 1e3, **over) -> dict:
    """Parameter set shared by all workloads: rho_l = 1000, rho_g = rho_l / ratio, mu 1e-3 / 1e-5 (App. B),
    eps = h, dt = 1e-4, c_mass = 1/dt, theta = 1/2 (Crank-Nicolson), dtau = min(eps, dt), variant 2."""
    h = L / n
    eps = h
    dt = 1e-4
    prm = dict(rho_l=1000.0, rho_g=1000.0 / ratio, mu_l=1e-3, mu_g=1e-5, eps=eps, dt=dt, c_mass=1.0 / dt,
               theta=0.5, dtau=min(eps, dt), variant=2, stress=1, corr_zone=0, newton=1, dirichlet_faces=0x3F,
               cpp_tol=1e-10, cpp_kmax=20, eta_n=2.0, eta_kappa=2.0)
    prm.update(over)
    return prm


def make_workload(name: str, n: int | None = None, p: int = 2, seed: int | None = None, **over) -> Workload:
    """Named workloads.

    sphere8   : 8^3, one sphere R = 0.25, ratio 1e3, mdot = 1, u0 then x ~ U[-1, 1] (seed 0)
    spheres64 : 64^3, four random spheres (seed 2), ratio 1e3, Fourier u0 (seed 2), x ~ U[-1, 1]
    slab96    : 96^3, slab at z = 0.5, ratio 1e3, Fourier u0 (seed 3), x plays the role of f ~ U[-1, 1] (seed 3)
    sphere48  : 48^3, sphere R = 0.25, w and x ~ U[-1,1] (seed 1), then u0 ~ U[-1, 1] (seed 1)
    deformed128: 128^3, deformed sphere (seed 5), ratio 1e4, Fourier u0 (seed 5)
    Any other n can be passed to reuse a recipe at a smaller size."""
    L = 1.0
    table = {
        "sphere8": dict(n=8, seed=0, geom="sphere", vel="uniform", ratio=1e3),
        "spheres64": dict(n=64, seed=2, geom="spheres", vel="fourier", ratio=1e3),
        "slab96": dict(n=96, seed=3, geom="slab", vel="fourier", ratio=1e3),
        "sphere48": dict(n=48, seed=1, geom="sphere", vel="uniform_after", ratio=1e3),
        "deformed128": dict(n=128, seed=5, geom="deformed", vel="fourier", ratio=1e4),
    }
    cfg = dict(table[name])
    if n is not None:
        cfg["n"] = n
    if seed is not None:
        cfg["seed"] = seed
    n = cfg["n"]
    rng = np.random.default_rng(cfg["seed"])
    prm = default_params(n, L, ratio=cfg["ratio"], **over)
    ns = int(prm.get("n_sub", 1))
    q1 = node_coords(ns * n, 1, L)  # level-set nodes
    d = signed_distance(cfg["geom"], q1, rng)
    phi = np.tanh(d / (2.0 * prm["eps"]))
    n_u = (p * n + 1) ** 3
    extra = {}
    if cfg["vel"] == "uniform":
        u0 = rng.uniform(-1.0, 1.0, 3 * n_u)
        x = rng.uniform(-1.0, 1.0, 3 * n_u)
    elif cfg["vel"] == "uniform_after":
        w = rng.uniform(-1.0, 1.0, 3 * n_u)
        x = rng.uniform(-1.0, 1.0, 3 * n_u)
        u0 = rng.uniform(-1.0, 1.0, 3 * n_u)
        extra["w"] = w
        extra["w_p"] = rng.uniform(-1.0, 1.0, (n + 1) ** 3)
    else:
        u0 = fourier_velocity(n, p, rng, L=L)
        x = rng.uniform(-1.0, 1.0, 3 * n_u)
    mdot = np.ones((ns * n + 1) ** 3)
    return Workload(n=n, p=p, L=L, params=prm, phi=phi, u0=u0, mdot=mdot, x=x, extra=extra)


def random_workload(n: int, p: int = 2, seed: int = 0, geom: str = "sphere", ratio: float = 1e3, **over) -> Workload:
    """Small random case for parity sweeps: given geometry, U[-1,1] velocity and applied vector, mdot ~ U[0.5, 1.5]."""
    L = 1.0
    rng = np.random.default_rng(seed)
    prm = default_params(n, L, ratio=ratio, **over)
    ns = int(prm.get("n_sub", 1))
    q1 = node_coords(ns * n, 1, L)  # level-set nodes
    d = signed_distance(geom, q1, rng)
    phi = np.tanh(d / (2.0 * prm["eps"]))
    n_u = (p * n + 1) ** 3
    u0 = rng.uniform(-1.0, 1.0, 3 * n_u)
    x = rng.uniform(-1.0, 1.0, 3 * n_u)
    mdot = rng.uniform(0.5, 1.5, (ns * n + 1) ** 3)
    return Workload(n=n, p=p, L=L, params=prm, phi=phi, u0=u0, mdot=mdot, x=x)
