"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test states the passage it checks.  A plausible mistake in the oracle (dropped term, wrong sign, transposed
index, wrong interpolation law) fails at least one of them:
  * closed forms of the material law (Eqs. heaviside, delta, rhoEff, muEff) and of the corrected strain
    (Eqs. 2d_example_eps / 2d_example_eps_eval, golden fixture);
  * the 1D evaporation pressure jump mdot^2 (1/rho_g - 1/rho_l) (Eqs. stefan_sharp_pressure /
    stefan_diffuse_pressure) reached by the reciprocal density, and the printed factor of 166 by which the
    arithmetic density overestimates it (Sec. 3.1.1, golden fixture);
  * exact integration of polynomial fields, zero viscous stress of rigid-body fields, zero corrected stress of a
    purely normal velocity on a flat interface (Sec. 2.4.2);
  * brute force: an independent per-quadrature-point loop over the weak form (App. D) with its own basis;
  * transport velocity: variant 1 vanishes exactly on the static flat interface (Sec. 2.3.4), variant 2 tends to
    zero, closest points lie on the isocontour phi = tanh(3/2) (App. C);
  * the hand-written adjoint gradients agree with central differences of the loss.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate

import workloads
from oracle import adjoint, fe, levelset, momentum, physics, solve, transport

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make_problem(n, p=2, phi=None, u0=None, mdot=None, rho_mode="reciprocal", **prm):
    mesh = fe.Mesh(n, p, 1.0)
    params = workloads.default_params(n)
    params.update(prm)
    phi = np.zeros(mesh.n_phi) if phi is None else phi
    u0 = np.zeros(3 * mesh.n_u) if u0 is None else u0
    mdot = np.ones(mesh.n_phi) if mdot is None else mdot
    return momentum.Problem(mesh=mesh, params=params, phi=phi, u0=u0, mdot=mdot, rho_mode=rho_mode)


def slab_phi(n, eps, z0=0.5):
    q1 = workloads.node_coords(n, 1)
    return np.tanh((z0 - q1[:, 2]) / (2 * eps))


# ---------------------------------------------------------------------------------------------------- material law
def test_heaviside_closed_forms():
    """Eq. (heaviside): H(0) = 1/2, H = 0 / 1 beyond -+3 eps, H(d) + H(-d) = 1, H continuous at the band edge."""
    eps = 0.1
    d = np.linspace(-0.4, 0.4, 161)
    phi = np.tanh(d / (2 * eps))
    H = physics.heaviside(phi, eps)
    assert physics.heaviside(np.array([0.0]), eps)[0] == 0.5
    assert np.all(H[d <= -3 * eps - 1e-12] == 0.0) and np.all(H[d >= 3 * eps + 1e-12] == 1.0)
    np.testing.assert_allclose(H + H[::-1], 1.0, atol=2e-15)
    inner = physics.heaviside(np.array([np.tanh(1.5 - 1e-9), -np.tanh(1.5 - 1e-9)]), eps)
    np.testing.assert_allclose(inner, [1.0, 0.0], atol=1e-12)
    # the zone boundary |phi| = tanh(3/2) is d = 3 eps (Eq. distance inverts Eq. initial_phi)
    assert abs(physics.distance(physics.PHI_BAND, eps) - 3 * eps) < 1e-14


def test_delta_normalisation():
    """Eq. (delta) keeps int_{-1}^{1} delta dphi = 1, i.e. int H'(d) dd = 1 over the interface zone."""
    eps = 0.05
    dH = lambda dd: physics.heaviside_parts(np.array([np.tanh(dd / (2 * eps))]), eps)[1][0]
    val, _ = scipy.integrate.quad(dH, -3 * eps, 3 * eps, limit=200)
    assert abs(val - 1.0) < 1e-10
    # in phi: dH/dphi = H'(d) d'(phi)
    f = lambda p: physics.heaviside_parts(np.array([p]), eps)[1][0] * physics.ddist_dphi(p, eps)
    val, _ = scipy.integrate.quad(f, -physics.PHI_BAND, physics.PHI_BAND, limit=200)
    assert abs(val - 1.0) < 1e-10


def test_delta_is_gradient_of_heaviside():
    """Eq. (delta): delta = |grad H(phi)| for a 1D profile phi(z), checked by differentiating H(phi(z)) numerically."""
    eps = 0.05
    z = np.linspace(0.35, 0.65, 31)
    phi = lambda zz: np.tanh((0.5 - zz) / (2 * eps))
    dphi = lambda zz: -(1 - np.tanh((0.5 - zz) / (2 * eps)) ** 2) / (2 * eps)
    g = np.zeros((z.size, 3))
    g[:, 2] = dphi(z)
    delta = physics.delta(phi(z), g, eps)
    hstep = 1e-6
    fd = np.abs(physics.heaviside(phi(z + hstep), eps) - physics.heaviside(phi(z - hstep), eps)) / (2 * hstep)
    np.testing.assert_allclose(delta, fd, rtol=1e-6, atol=1e-8)


def test_density_viscosity_closed_forms():
    """Eqs. (rhoEff), (muEff): end values, 1/rho affine in H, local mass conservation rho (mdot/rho) = mdot."""
    H = np.linspace(0.0, 1.0, 101)
    rho = physics.density(H, 1000.0, 1.0)
    assert rho[0] == 1.0 and rho[-1] == 1000.0
    np.testing.assert_allclose(np.diff(1.0 / rho, 2), 0.0, atol=1e-15)
    mdot = 0.37
    np.testing.assert_allclose(rho * (mdot / rho), mdot, rtol=2e-16)
    mu = physics.viscosity(H, 1e-3, 1e-5)
    assert mu[0] == 1e-5 and mu[-1] == 1e-3
    ra = physics.density(H, 1000.0, 1.0, mode="arithmetic")
    np.testing.assert_allclose(np.diff(ra, 2), 0.0, atol=1e-9)


def test_corrected_strain_shell_example():
    """Eq. (2d_example_eps_eval): diag(a, b) - (a + b) e1 (x) e1 = diag(-b, b) (golden fixture)."""
    fx = json.load(open(os.path.join(GOLDEN, "shell_strain.json")))
    for case in fx["cases"]:
        e = np.diag([case["a"], case["b"]])
        out = physics.corrected_strain(e, np.array([1.0, 0.0]), True)
        np.testing.assert_allclose(out, case["expected"], atol=1e-15)
    rng = np.random.default_rng(3)
    for _ in range(10):
        G = rng.standard_normal((3, 3))
        e = 0.5 * (G + G.T)
        nv = rng.standard_normal(3)
        nv /= np.linalg.norm(nv)
        assert abs(np.trace(physics.corrected_strain(e, nv, True))) < 1e-14  # deviatoric, Sec. 2.4.2


# ------------------------------------------------------------------------------------------- operator closed forms
def _convection_sum(n, rho_mode):
    """Sum over the z-rows of rho (u.grad) u for u = (mdot/rho_recip) e_z on a slab (Picard, no mass/viscosity)."""
    eps = 0.1
    pb = make_problem(n, phi=slab_phi(n, eps), rho_mode=rho_mode, eps=eps, rho_l=1.0, rho_g=1e-3, c_mass=0.0,
                      mu_l=0.0, mu_g=0.0, newton=0, dirichlet_faces=0)
    mesh = pb.mesh
    # phi_h at the Q2 nodes (trilinear interpolation of the Q1 level set), then u = mdot / rho(phi_h)
    zq = workloads.node_coords(n, 2)[:, 2]
    q1z = workloads.node_coords_1d(n, 1)
    phin = np.interp(zq, q1z, np.tanh((0.5 - q1z) / (2 * eps)))     # phi_h along z (trilinear = linear in z)
    uz = 1.0 / physics.density(physics.heaviside(phin, eps), 1.0, 1e-3)
    u = np.zeros(3 * mesh.n_u)
    u[2 * mesh.n_u:] = uz
    pb.u0 = u
    y = momentum.assemble(pb) @ u
    return y[2 * mesh.n_u:].sum()


def test_pressure_jump_reciprocal_density():
    """Eqs. (stefan_sharp_pressure)/(stefan_diffuse_pressure): the momentum flux balance across a flat evaporating
    interface, int rho u du/dz = mdot (u_g - u_l) = mdot^2 (1/rho_g - 1/rho_l), holds for the reciprocal density
    (rho u = mdot pointwise) and converges with mesh refinement."""
    exact = 1.0 * (1.0 / 1e-3 - 1.0)
    errs = [abs(_convection_sum(n, "reciprocal") - exact) / exact for n in (6, 12)]
    assert errs[1] < errs[0]
    assert errs[1] < 2e-2


def test_pressure_overestimate_arithmetic_density():
    """Sec. 3.1.1: an arithmetic density overestimates the liquid pressure by the printed factor 166; the closed
    form of the ratio is int_0^1 (H r + 1 - H)(H + (1 - H) r) / r dH = 2/3 + (r + 1/r)/6 = 167.33 for r = 1000."""
    fx = json.load(open(os.path.join(GOLDEN, "pressure_jump_1d.json")))
    r = fx["rho_l"] / fx["rho_g"]
    closed = 2.0 / 3.0 + (r + 1.0 / r) / 6.0
    assert abs((closed - 1.0) - fx["printed_overestimate_factor"]) < 0.5
    n = 12
    ratio = _convection_sum(n, "arithmetic") / _convection_sum(n, "reciprocal")
    assert abs(ratio - closed) / closed < 3e-2


def test_rigid_body_has_no_viscous_stress():
    """Eq. (stokesLaw)/(modified_viscous_stress): eps(a + w x X) = 0, so the viscous operator annihilates rigid
    motions for either stress law and any level set (mass and convection switched off, no Dirichlet rows)."""
    wl = workloads.random_workload(3, seed=4, geom="sphere")
    X = workloads.node_coords(3, 2)
    a, w = np.array([0.3, -1.1, 0.7]), np.array([0.5, 0.2, -0.9])
    x = (a[None] + np.cross(w[None], X)).T.ravel()
    for stress, zone in ((0, 0), (1, 0), (1, 1)):
        pb = make_problem(3, phi=wl.phi, c_mass=0.0, dirichlet_faces=0, stress=stress, corr_zone=zone,
                          eps=wl.params["eps"])
        A = momentum.assemble(pb)
        scale = np.abs(A).sum(axis=1).max() * np.abs(x).max()
        assert np.abs(A @ x).max() < 1e-13 * scale


def test_corrected_stress_flat_interface():
    """Sec. 2.4.2 / 3.1.2: for a flat interface n = e_z and x = f(z) e_z the corrected strain vanishes, so the
    corrected viscous operator gives zero while the standard Stokes law does not (the pressure artifact)."""
    n, eps = 4, 0.15
    pb = make_problem(n, phi=slab_phi(n, eps), c_mass=0.0, dirichlet_faces=0, stress=1, corr_zone=1, eps=eps)
    zq = workloads.node_coords(n, 2)[:, 2]
    x = np.zeros(3 * pb.mesh.n_u)
    x[2 * pb.mesh.n_u:] = np.sin(3.0 * zq) + zq ** 2
    A = momentum.assemble(pb)
    scale = np.abs(A).sum(axis=1).max() * np.abs(x).max()
    assert np.abs(A @ x).max() < 1e-13 * scale
    pb.params["stress"] = 0
    assert np.abs(momentum.assemble(pb) @ x).max() > 1e-3 * scale


def test_exact_integration_constant_phase():
    """Constant phase (H = 1): the Q2 Gauss rule integrates polynomial fields exactly (Sec. 2.5):
    1^T M 1 = rho c_m |Omega|, x^T M x = rho c_m int x^2, x^T K x = 2 mu |sym G|^2 for x = G X."""
    n = 3
    prm = dict(dirichlet_faces=0, rho_l=7.0, mu_l=0.3)
    phi1 = np.ones((n + 1) ** 3)
    X = workloads.node_coords(n, 2)
    pb = make_problem(n, phi=phi1, **prm)
    A = momentum.assemble(pb)
    Nu = pb.mesh.n_u
    ones = np.zeros(3 * Nu)
    ones[Nu:2 * Nu] = 1.0
    np.testing.assert_allclose((A @ ones)[Nu:2 * Nu].sum(), 7.0 * pb.params["c_mass"], rtol=1e-13)
    f = 1.0 + X[:, 0] + 2.0 * X[:, 1] ** 2 - X[:, 0] * X[:, 2]
    xq = np.zeros(3 * Nu)
    xq[:Nu] = f
    t, wts = np.polynomial.legendre.leggauss(6)
    t, wts = 0.5 * (t + 1), 0.5 * wts
    T = np.meshgrid(t, t, t, indexing="ij")
    Wt = np.einsum("i,j,k->ijk", wts, wts, wts)
    fint = np.sum(Wt * (1.0 + T[0] + 2.0 * T[1] ** 2 - T[0] * T[2]) ** 2)
    pbm = make_problem(n, phi=phi1, mu_l=0.0, mu_g=0.0, dirichlet_faces=0, rho_l=7.0)
    np.testing.assert_allclose(xq @ (momentum.assemble(pbm) @ xq), 7.0 * pbm.params["c_mass"] * fint, rtol=1e-12)
    G = np.array([[0.2, -1.0, 0.5], [0.7, 0.1, 0.0], [-0.3, 0.4, -0.6]])
    xl = (X @ G.T).T.ravel()
    pbk = make_problem(n, phi=phi1, c_mass=0.0, dirichlet_faces=0, mu_l=0.3)
    S = 0.5 * (G + G.T)
    np.testing.assert_allclose(xl @ (momentum.assemble(pbk) @ xl), 2 * 0.3 * np.sum(S * S), rtol=1e-12)


def test_convection_and_newton_terms():
    """Weak convection (u0.grad)x and Newton term (x.grad)u0 (App. D): for u0 = a, x = (b.X) e_c the rows of
    component c sum to rho a.b; for u0 = G0 X, x = e_d they sum to rho G0[:, d] (test functions sum to one)."""
    n = 2
    X = workloads.node_coords(n, 2)
    phi1 = np.ones((n + 1) ** 3)
    base = dict(c_mass=0.0, mu_l=0.0, mu_g=0.0, dirichlet_faces=0, rho_l=3.0)
    a, b = np.array([0.4, -0.2, 1.5]), np.array([-1.0, 2.0, 0.5])
    pb = make_problem(n, phi=phi1, u0=np.repeat(a, X.shape[0]), **base)
    Nu = pb.mesh.n_u
    x = np.zeros(3 * Nu)
    x[Nu:2 * Nu] = X @ b
    y = momentum.assemble(pb) @ x
    np.testing.assert_allclose([y[:Nu].sum(), y[Nu:2 * Nu].sum(), y[2 * Nu:].sum()], [0, 3.0 * a @ b, 0], atol=1e-12)
    G0 = np.array([[0.2, -1.0, 0.5], [0.7, 0.1, 0.0], [-0.3, 0.4, -0.6]])
    pb = make_problem(n, phi=phi1, u0=(X @ G0.T).T.ravel(), **base)
    for d in range(3):
        x = np.zeros(3 * Nu)
        x[d * Nu:(d + 1) * Nu] = 1.0
        y = momentum.assemble(pb) @ x
        np.testing.assert_allclose([y[:Nu].sum(), y[Nu:2 * Nu].sum(), y[2 * Nu:].sum()], 3.0 * G0[:, d], atol=1e-12)
    pb.params["newton"] = 0
    y = momentum.assemble(pb) @ x
    np.testing.assert_allclose([y[:Nu].sum(), y[Nu:2 * Nu].sum(), y[2 * Nu:].sum()], 0.0, atol=1e-12)


def test_divergence_row():
    """First line of Eq. (weakNavierStokes): (q, div x) = (q, v_dil).  For x = X, sum_j y_p[j] = 3 - int v_dil;
    without evaporation exactly 3; on a flat interface int v_dil -> mdot (1/rho_g - 1/rho_l) since int delta dz = 1
    (the sign of App. A: div u = mdot (1/rho_g - 1/rho_l) delta, evaporation expands the volume)."""
    n = 4
    X = workloads.node_coords(n, 2)
    x = X.T.ravel().copy()
    pb = make_problem(n, phi=slab_phi(n, 0.1), mdot=np.zeros((n + 1) ** 3), dirichlet_faces=0, eps=0.1)
    B, g = momentum.divergence(pb)
    np.testing.assert_allclose((B @ x - g).sum(), 3.0, rtol=1e-13)
    kr = 1.0 / 1.0 - 1.0 / 1000.0
    errs = []
    for n in (8, 16):
        X = workloads.node_coords(n, 2)
        pb = make_problem(n, phi=slab_phi(n, 0.1), dirichlet_faces=0, eps=0.1)
        B, g = momentum.divergence(pb)
        errs.append(abs((B @ X.T.ravel() - g).sum() - (3.0 - kr)) / abs(kr))
    assert errs[1] < errs[0] and errs[1] < 5e-3


def test_levelset_operators_closed_forms():
    """Q1 operators of Eqs. (weakFormLevelSet) and (reinitialization) on polynomial fields."""
    n = 3
    mesh = fe.Mesh(n, 1, 1.0)
    X = workloads.node_coords(n, 1)
    a, b = np.array([0.3, -0.8, 1.2]), np.array([1.0, 0.5, -2.0])
    theta, dt = 0.5, 0.01
    A = levelset.advection_matrix(mesh, np.repeat(a, X.shape[0]), theta, dt)
    np.testing.assert_allclose((A @ np.ones(mesh.n_phi)).sum(), 1.0, rtol=1e-14)
    xl = X @ b
    np.testing.assert_allclose((A @ xl).sum(), b @ np.full(3, 0.5) + theta * dt * (a @ b), rtol=1e-13)
    phi_lin = 0.8 * (X[:, 2] - 0.5)               # grad phi = 0.8 e_z -> n = e_z everywhere
    eps, dtau = 0.05, 0.02
    R = levelset.reinit_matrix(mesh, phi_lin, eps, dtau)
    int_sq = np.sum(b * b) / 3.0 + (np.sum(b) ** 2 - np.sum(b * b)) / 4.0
    np.testing.assert_allclose(xl @ (R @ xl), int_sq / dtau + eps * b[2] ** 2, rtol=1e-13)
    r = levelset.reinit_rhs(mesh, phi_lin, np.full(mesh.n_phi, 0.4), dtau)
    np.testing.assert_allclose(r.sum(), 0.4 / dtau, rtol=1e-13)
    # compressive flux (grad w, (1 - psi^2)/2 n) for psi = 0: sum over a test function gradient w = z gives 1/2
    r0 = levelset.reinit_rhs(mesh, phi_lin, np.zeros(mesh.n_phi), dtau)
    np.testing.assert_allclose(r0 @ X[:, 2], 0.5, rtol=1e-13)


# ------------------------------------------------------------------------------------------------- brute force
def _basis_1d(nodes):
    """Lagrange basis through ``nodes`` as power-series coefficients (Vandermonde inverse), independent of oracle.fe."""
    V = np.vander(nodes, increasing=True)
    coef = np.linalg.inv(V)                                     # column a: coefficients of l_a
    polys = [np.polynomial.Polynomial(coef[:, a]) for a in range(len(nodes))]
    return polys, [p.deriv() for p in polys]


def _naive_apply(wl_n, p, prm, phi, u0, mdot, x, w_p=None):
    """y = A x and y_p = B x - g by a per-cell, per-quadrature-point loop written from the weak form (App. D)."""
    n = wl_n
    h = 1.0 / n
    m = p * n + 1
    Nu = m ** 3
    gl = {2: [0.0, 0.5, 1.0], 3: [0.0, 0.5 - 0.5 / math.sqrt(5), 0.5 + 0.5 / math.sqrt(5), 1.0]}[p]
    L, dL = _basis_1d(np.array(gl))
    L1, dL1 = _basis_1d(np.array([0.0, 1.0]))
    t, wq = np.polynomial.legendre.leggauss(p + 1)
    t, wq = 0.5 * (t + 1), 0.5 * wq
    y = np.zeros(3 * Nu)
    yp = np.zeros((n + 1) ** 3)
    eps = prm["eps"]
    for cz in range(n):
        for cy in range(n):
            for cx in range(n):
                loc = [(a, b, c) for c in range(p + 1) for b in range(p + 1) for a in range(p + 1)]
                gidx = [(p * cx + a) + m * ((p * cy + b) + m * (p * cz + c)) for (a, b, c) in loc]
                loc1 = [(a, b, c) for c in range(2) for b in range(2) for a in range(2)]
                gidx1 = [(cx + a) + (n + 1) * ((cy + b) + (n + 1) * (cz + c)) for (a, b, c) in loc1]
                for qz in range(p + 1):
                    for qy in range(p + 1):
                        for qx in range(p + 1):
                            s = (t[qx], t[qy], t[qz])
                            W = wq[qx] * wq[qy] * wq[qz] * h ** 3
                            Nv = [L[a](s[0]) * L[b](s[1]) * L[c](s[2]) for (a, b, c) in loc]
                            Ng = [np.array([dL[a](s[0]) * L[b](s[1]) * L[c](s[2]), L[a](s[0]) * dL[b](s[1]) * L[c](s[2]),
                                            L[a](s[0]) * L[b](s[1]) * dL[c](s[2])]) / h for (a, b, c) in loc]
                            M1 = [L1[a](s[0]) * L1[b](s[1]) * L1[c](s[2]) for (a, b, c) in loc1]
                            G1 = [np.array([dL1[a](s[0]) * L1[b](s[1]) * L1[c](s[2]), L1[a](s[0]) * dL1[b](s[1]) * L1[c](s[2]),
                                            L1[a](s[0]) * L1[b](s[1]) * dL1[c](s[2])]) / h for (a, b, c) in loc1]
                            ph = sum(M1[j] * phi[gidx1[j]] for j in range(8))
                            gph = sum(G1[j] * phi[gidx1[j]] for j in range(8))
                            md = sum(M1[j] * mdot[gidx1[j]] for j in range(8))
                            U = np.array([sum(Nv[i] * u0[c * Nu + gidx[i]] for i in range(len(loc))) for c in range(3)])
                            GU = np.array([sum(Ng[i] * u0[c * Nu + gidx[i]] for i in range(len(loc))) for c in range(3)])
                            Xv = np.array([sum(Nv[i] * x[c * Nu + gidx[i]] for i in range(len(loc))) for c in range(3)])
                            GX = np.array([sum(Ng[i] * x[c * Nu + gidx[i]] for i in range(len(loc))) for c in range(3)])
                            # material law at the point
                            if abs(ph) < math.tanh(1.5):
                                d = eps * math.log((1 + ph) / (1 - ph))
                                H = 0.5 + d / (6 * eps) + math.sin(math.pi * d / (3 * eps)) / (2 * math.pi)
                                dH = (1 + math.cos(math.pi * d / (3 * eps))) / (6 * eps)
                                delta = dH * 2 * eps / (1 - ph * ph) * np.linalg.norm(gph)
                                zone = True
                            else:
                                H, delta, zone = (1.0 if ph > 0 else 0.0), 0.0, False
                            rho = 1.0 / (H / prm["rho_l"] + (1 - H) / prm["rho_g"])
                            mu = H * prm["mu_l"] + (1 - H) * prm["mu_g"]
                            gn = np.linalg.norm(gph)
                            nv = gph / gn if gn > 0 else np.zeros(3)
                            F = rho * (prm["c_mass"] * Xv + GX @ U + prm["newton"] * (GU @ Xv))
                            E = 0.5 * (GX + GX.T)
                            zz = (prm["stress"] == 1) and (zone or prm["corr_zone"] == 1)
                            if zz:
                                E = E - np.trace(GX) * np.outer(nv, nv)
                            T = 2 * mu * E
                            for i in range(len(loc)):
                                for c in range(3):
                                    y[c * Nu + gidx[i]] += W * (Nv[i] * F[c] + Ng[i] @ T[c])
                            vdil = md * (1 / prm["rho_g"] - 1 / prm["rho_l"]) * delta  # App. A sign of Eq. (evaporDil)
                            for j in range(8):
                                yp[gidx1[j]] += W * M1[j] * (np.trace(GX) - vdil)
    return y, yp


@pytest.mark.parametrize("n,p,geom,stress,zone,newton", [(1, 2, "sphere", 1, 0, 1), (2, 2, "sphere", 1, 0, 1),
                                                          (2, 2, "slab", 0, 0, 0), (2, 2, "sphere", 1, 1, 1),
                                                          (1, 3, "sphere", 1, 0, 1)])
def test_brute_force_small_meshes(n, p, geom, stress, zone, newton):
    """Oracle assembly against the naive per-point loop on 1 and 2^3 cells (Dirichlet off, random fields)."""
    wl = workloads.random_workload(n, p=p, seed=11 + n, geom=geom, ratio=1e3, dirichlet_faces=0, stress=stress,
                                   corr_zone=zone, newton=newton)
    wl.params["eps"] = 0.25
    rng = np.random.default_rng(5)
    wl.phi = rng.uniform(-0.95, 0.95, wl.phi.shape)  # many points inside the interface zone
    pb = momentum.Problem.from_workload(wl)
    y, yp = momentum.apply(pb, wl.x, with_divergence=True)
    yn, ypn = _naive_apply(n, p, wl.params, wl.phi, wl.u0, wl.mdot, wl.x)
    np.testing.assert_allclose(y, yn, rtol=1e-12, atol=1e-12 * np.abs(yn).max())
    np.testing.assert_allclose(yp, ypn, rtol=1e-12, atol=1e-12 * np.abs(ypn).max())


def test_sampled_rows_match_full_apply():
    """oracle.momentum.apply_rows (cells around sampled nodes only) equals rows of the assembled product."""
    wl = workloads.random_workload(4, seed=2)
    pb = momentum.Problem.from_workload(wl)
    y = momentum.apply(pb, wl.x)
    nodes = np.array([0, 7, 40, 100, pb.mesh.n_u - 1, 365])
    yr = momentum.apply_rows(pb, wl.x, nodes)
    for c in range(3):
        np.testing.assert_allclose(yr[c], y[c * pb.mesh.n_u + nodes], rtol=1e-13, atol=1e-10)


def test_dirichlet_rows_identity():
    """Constrained velocity DoFs: y = x there, and x there does not enter other rows."""
    wl = workloads.random_workload(3, seed=9)
    pb = momentum.Problem.from_workload(wl)
    mask = pb.constrained()
    y = momentum.apply(pb, wl.x)
    np.testing.assert_array_equal(y[mask], wl.x[mask])
    x2 = wl.x.copy()
    x2[mask] += 5.0
    np.testing.assert_allclose(momentum.apply(pb, x2)[~mask], y[~mask], rtol=1e-14, atol=1e-9)


# --------------------------------------------------------------------------------------------- transport velocity
def _flat_static(n, eps, variant, rho_l=1000.0, rho_g=1.0):
    """Flat interface, inflow mdot/rho_l: the diffuse velocity is u = mdot/rho(H) e_z (Eq. stefan_diffuse_velocity
    with u_bar = mdot/rho_l, liquid below), so the exact transport velocity vanishes (Sec. 2.3.4)."""
    mesh = fe.Mesh(n, 2, 1.0)
    prm = workloads.default_params(n, eps=eps, variant=variant, rho_l=rho_l, rho_g=rho_g)
    phi = slab_phi(n, eps)
    zq = workloads.node_coords(n, 2)[:, 2]
    phin = np.tanh((0.5 - zq) / (2 * eps))           # equals the nodal level set where a Q2 node is a Q1 node
    u0 = np.zeros(3 * mesh.n_u)
    u0[2 * mesh.n_u:] = 1.0 / physics.density(physics.heaviside(phin, eps), rho_l, rho_g)
    ug, flags = transport.transport_velocity(mesh, phi, u0, np.ones(mesh.n_phi), prm)
    return ug, flags, phi


def test_transport_velocity_variant1_flat_is_zero():
    """Variant 1, Eq. (transport_vel_local_continuous): u + mdot/rho n = 0 at every node of the static flat case."""
    ug, flags, _ = _flat_static(4, 0.1, 1)
    assert np.abs(ug).max() < 1e-15 and flags.sum() == 0


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("rho_g", [0.5, 1e-3])
def test_transport_velocity_extension_flat_is_small(variant, rho_g):
    """Variants 2/3, Eqs. (transport_vel_extension_liquid)/(transport_vel_extension_gas): on the static flat interface
    u(x_l) + mdot/rho_l n and u(x_g) + mdot/rho_g n vanish up to the interpolation error of u at the projected point,
    far below the velocity jump mdot (1/rho_g - 1/rho_l); a sign error, the other phase's density or the wrong
    isocontour would each leave an error of the order of the jump or of mdot/rho."""
    for n in (4, 8, 16):
        ug, flags, phi = _flat_static(n, 0.1, variant, rho_l=1.0, rho_g=rho_g)
        assert flags.sum() == 0
        np.testing.assert_allclose(ug[:2], 0.0, atol=1e-14)
        jump = 1.0 / rho_g - 1.0
        assert np.abs(ug[2]).max() < 1e-3 * jump


def test_closest_points_on_isocontour():
    """App. C, Eq. (cpp): closest points lie on phi_h = tanh(+-3/2) and are (up to the discrete isocontour's kinks)
    the nearest such points: |y - x| exceeds a brute-force minimum over points of the isocontour, found by bisection
    along rays from the sphere centre, by at most 0.3 cells.  At most 5 % of the nodes may end flagged."""
    n = 12
    mesh = fe.Mesh(n, 2, 1.0)
    eps = mesh.h
    q1 = workloads.node_coords(n, 1)
    m1 = n + 1
    c = np.full(3, 0.5 * n)
    dirs = np.random.default_rng(0).standard_normal((3000, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    # variant-2 target inside a large droplet, variant-3 target around a small one (both contours inside the box)
    for target, level, radius, lo_phi, hi_phi in ((3 * eps, physics.PHI_BAND, 0.4, -math.tanh(3.0), physics.PHI_BAND),
                                                  (-3 * eps, -physics.PHI_BAND, 0.2, -physics.PHI_BAND, math.tanh(3.0))):
        phi = np.tanh(workloads.signed_distance("sphere", q1, radius=radius) / (2 * eps))
        ev = transport.PointEval(mesh, phi, np.zeros(3 * mesh.n_u))
        nodes = [k for k in range(mesh.n_phi) if lo_phi < phi[k] < hi_phi][::9]
        assert len(nodes) > 20
        samples = []
        for dv in dirs:
            lo, hi = 0.0, 0.49 * n
            for _ in range(40):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if ev.phi_grad(c + mid * dv)[0] > level else (lo, mid)
            samples.append(c + lo * dv)
        samples = np.array(samples)
        cosines = []
        n_ok = 0
        for node in nodes:
            sx = np.array([node % m1, (node // m1) % m1, node // (m1 * m1)], dtype=float)
            y, ok = transport.closest_point(ev, sx, target, eps, 1e-10, 50)
            if not ok:   # descent stalled on a crease of the discrete isocontour: flagged, not checked
                continue
            n_ok += 1
            ph, g = ev.phi_grad(y)
            assert abs(physics.distance(ph, eps) - target) < 1e-9 * mesh.h
            dmin = np.min(np.linalg.norm(samples - sx, axis=1))
            assert np.linalg.norm(y - sx) <= dmin + 0.3
            if np.linalg.norm(y - sx) > 0.5:
                cosines.append(abs((y - sx) @ g) / (np.linalg.norm(y - sx) * np.linalg.norm(g)))
        assert np.median(cosines) > 0.9
        assert n_ok >= 0.95 * len(nodes)


# ------------------------------------------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("stress,zone,newton", [(1, 0, 1), (0, 0, 0), (1, 1, 1)])
def test_adjoint_gradients_match_central_differences(stress, zone, newton):
    """Hand-written chain rule (rhoEff, muEff, delta, normal_vector, corrected strain) against central differences of
    L = w.A x + w_p.(B x - g)."""
    n = 3
    wl = workloads.random_workload(n, seed=21, geom="sphere", stress=stress, corr_zone=zone, newton=newton)
    wl.params["eps"] = 0.2
    rng = np.random.default_rng(8)
    wl.phi = rng.uniform(-0.85, 0.85, wl.phi.shape)
    pb = momentum.Problem.from_workload(wl)
    w = rng.uniform(-1, 1, wl.x.shape)
    w_p = rng.uniform(-1, 1, wl.phi.shape)
    g_u0, g_phi, g_mdot = adjoint.param_gradients(pb, wl.x, w, w_p)
    gx = adjoint.grad_x(pb, w, w_p)

    def L(**kw):
        q = momentum.Problem(mesh=pb.mesh, params=pb.params, phi=kw.get("phi", pb.phi), u0=kw.get("u0", pb.u0),
                             mdot=kw.get("mdot", pb.mdot))
        return adjoint.loss(q, kw.get("x", wl.x), w, w_p)

    for name, g, base, t in (("phi", g_phi, pb.phi, 1e-6), ("mdot", g_mdot, pb.mdot, 1e-3),
                             ("u0", g_u0, pb.u0, 1e-3), ("x", gx, wl.x, 1e-3)):
        for k in range(3):
            v = rng.standard_normal(base.shape)
            fd = (L(**{name: base + t * v}) - L(**{name: base - t * v})) / (2 * t)
            an = g @ v
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.abs(g).sum()), (name, fd, an)


def test_direct_solve_residual():
    """oracle.solve is the definition x = A^{-1} f: its residual is at round-off level."""
    wl = workloads.make_workload("sphere8", n=4)
    pb = momentum.Problem.from_workload(wl)
    f = wl.x
    x = solve.solve(pb, f)
    r = momentum.assemble(pb) @ x - f
    assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-12


def test_closest_point_rounding_sensitivity():
    """Documents the resolution of the closest-point iteration (App. C reading): perturbing phi by ~1 ulp moves
    only a small fraction of the converged nodes, most of them by less than 1e-6 (the stopping decision is taken
    at rounding level near the minimum; a few nodes on creases of the discrete isocontour switch local minima)."""
    n = 12
    wl = workloads.random_workload(n, seed=5, geom="sphere", variant=2)
    q1 = workloads.node_coords(n, 1)
    wl.phi = np.tanh(workloads.signed_distance("sphere", q1, radius=0.3) / (2 * wl.params["eps"]))
    mesh = fe.Mesh(n, 2, 1.0)
    ug, fl = transport.transport_velocity(mesh, wl.phi, wl.u0, wl.mdot, wl.params)
    rng = np.random.default_rng(1)
    phi2 = wl.phi * (1 + 2e-16 * rng.standard_normal(wl.phi.shape))
    ug2, fl2 = transport.transport_velocity(mesh, phi2, wl.u0, wl.mdot, wl.params)
    ok = (fl == 0) & (fl2 == 0)
    d = np.abs(ug - ug2).max(axis=0)[ok]
    assert np.mean(fl == fl2) >= 0.98
    assert np.mean(d <= 1e-6 * np.abs(ug).max()) >= 0.99


@pytest.mark.parametrize("name", ["sphere8", "spheres64", "sphere48", "slab96", "deformed128"])
def test_normal_cutoff_is_inactive_near_the_interface(name):
    """The reading that sets n = 0 where |grad phi_h| h <= 1e-4 (physics.has_normal) changes nothing where the normal
    matters: on every workload (phi = tanh(d / 2 eps), eps = h) |grad phi_h| h exceeds the cut-off at every velocity
    quadrature point of the interface zone |phi_h| < tanh(3/2) (where the corrected stress and the delta use n) and at
    every Q1 node of the closest-point band -tanh(3) < phi < tanh(3) of variants 2 and 3 (n(x) of the transport
    velocity), by a margin of at least 10.  (For the tanh profile |grad phi| h = (1 - phi^2) |grad d| h / (2 eps), at
    least 0.09 in the zone and 0.005 at the band edge; the cut-off acts only ~9 eps or more from an interface.)"""
    wl = workloads.make_workload(name)
    mesh = fe.Mesh(wl.n, 1, wl.L)
    h = mesh.h
    assert wl.params["eps"] == pytest.approx(h)
    t, _ = fe.gauss_rule(wl.p + 1)
    b1 = fe.tensor_basis(1, t, h)
    cells = mesh.cells()
    worst = np.inf
    for s in range(0, len(cells), 65536):
        ph = wl.phi[mesh.dofs_phi(cells[s:s + 65536])]                 # [nc, 8]
        pq = ph @ b1.N                                                 # [nc, nq]
        gq = np.linalg.norm(np.einsum("nj,bjq->nqb", ph, b1.G), axis=-1)
        zone = physics.in_zone(pq)
        if zone.any():
            assert np.all(physics.has_normal(gq[zone], h))
            worst = min(worst, float(gq[zone].min() * h))
    # node gradients as the transport velocity takes them: the point-located cell's trilinear interpolant at the node
    m1 = wl.n + 1
    P = wl.phi.reshape(m1, m1, m1)                                     # [z, y, x]
    band = (-physics.PHI_GAS_BAND < P) & (P < physics.PHI_GAS_BAND)
    g = np.zeros((3,) + P.shape)
    for ax, axis in ((0, 2), (1, 1), (2, 0)):                          # x, y, z derivative along array axes 2, 1, 0
        fwd = np.diff(P, axis=axis) / h                                # cell of the node = floor, clamped to n - 1
        last = np.take(fwd, [-1], axis=axis)
        g[ax] = np.concatenate([fwd, last], axis=axis)
    # the trilinear gradient at a cell corner is the edge difference along that axis (the other coordinates at the
    # corner), so the node's gradient is the forward difference (backward on the last node)
    gn = np.linalg.norm(g, axis=0)
    assert np.all(physics.has_normal(gn[band], h))
    worst = min(worst, float(gn[band].min() * h))
    assert worst > 10 * physics.GRAD_TINY, worst
