"""Pins of the oracle's surface-tension force (Eq. surfaceTension with the density-scaled delta) against closed
forms and invariants.  CPU only."""
import numpy as np
import pytest

import workloads
from oracle import fe, momentum, physics, surface


def test_density_scaled_delta_integrates_to_one():
    """Across an interface with the equilibrium profile phi = tanh(d / (2 eps)), delta = H'(d) and
    int delta rho(H) c_rho dd = c_rho int_0^1 rho(H) dH = 1 for the reciprocal rho (the purpose of c_rho)."""
    for rho_l, rho_g in [(1000.0, 1.0), (1000.0, 0.1), (2.0, 1.0)]:
        eps = 0.01
        d = np.linspace(-3 * eps, 3 * eps, 400001)
        phi = np.tanh(d / (2 * eps))
        grad = np.zeros((d.size, 3))
        grad[:, 2] = (1 - phi ** 2) / (2 * eps)   # d phi / d z for phi(z) = tanh(z / (2 eps))
        dr = surface.density_scaled_delta(phi, grad, eps, rho_l, rho_g)
        val = np.sum(0.5 * (dr[1:] + dr[:-1]) * np.diff(d))
        assert val == pytest.approx(1.0, rel=1e-6), (rho_l, rho_g)


def _slab_problem(n, eps_cells=1.5):
    wl = workloads.random_workload(n, 2, 3, geom="slab", dirichlet_faces=0)
    mesh = fe.Mesh(n, 2, 1.0)
    prm = dict(wl.params)
    prm["eps"] = eps_cells / n
    r = np.arange(n + 1) / n
    Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
    phi = np.tanh((0.5 - Z.ravel()) / (2 * prm["eps"]))
    pb = momentum.Problem(mesh=mesh, params=prm, phi=phi, u0=wl.u0, mdot=wl.mdot)
    return pb, mesh


def test_slab_force_is_alpha_kappa_times_area():
    """Flat interface z = 1/2 with uniform kappa and n = -e_z (liquid below): sum_i b_(i,z) = -alpha kappa int delta_rho
    dV = -alpha kappa (unit cross-section; the x, y components vanish; the discrete delta integrates to 0.991 with
    eps = 1.5 h, the Q1 interpolant of the 3-cell-wide profile: a quadrature error that does not depend on h at fixed
    eps / h)."""
    pb, mesh = _slab_problem(16)
    nf = np.zeros((3, mesh.n_phi))
    nf[2] = -1.0
    kappa = np.full(mesh.n_phi, 3.0)
    alpha = 0.07
    b = surface.surface_tension_rhs(pb, nf, kappa, alpha).reshape(3, -1)
    assert np.abs(b[0]).max() == 0.0 and np.abs(b[1]).max() == 0.0
    assert b[2].sum() == pytest.approx(-alpha * 3.0, rel=2e-2)


def test_sphere_net_force_vanishes_and_points_inward():
    """A spherical drop with the curvature field 2/R and the radial normal: the force density points into the
    liquid (inward), and by symmetry the net force is zero to rounding relative to its total magnitude."""
    n = 12
    wl = workloads.random_workload(n, 2, 2, geom="sphere", dirichlet_faces=0)
    pb = momentum.Problem.from_workload(wl)
    mesh = pb.mesh
    r1 = np.arange(n + 1) / n
    Z, Y, X = np.meshgrid(r1, r1, r1, indexing="ij")
    rv = np.stack([X.ravel() - 0.5, Y.ravel() - 0.5, Z.ravel() - 0.5])
    rn = np.maximum(np.linalg.norm(rv, axis=0), 1e-12)
    nf = -rv / rn                                    # into the liquid drop
    kappa = np.full(mesh.n_phi, 2.0 / 0.25)
    b = surface.surface_tension_rhs(pb, nf, kappa, 1.0).reshape(3, -1)
    tot = np.abs(b).sum()
    assert tot > 0
    assert np.abs(b.sum(axis=1)).max() < 1e-12 * tot
    m = mesh.m
    g = np.arange(m) / (m - 1)
    Zu, Yu, Xu = np.meshgrid(g, g, g, indexing="ij")
    radial = np.stack([Xu.ravel() - 0.5, Yu.ravel() - 0.5, Zu.ravel() - 0.5])
    assert np.sum(b * radial) < 0.0


def test_constrained_entries_are_zero():
    wl = workloads.random_workload(6, 2, 4, geom="sphere")
    pb = momentum.Problem.from_workload(wl)
    nf = np.ones((3, pb.mesh.n_phi))
    b = surface.surface_tension_rhs(pb, nf, np.ones(pb.mesh.n_phi), 1.0)
    assert np.all(b[pb.constrained()] == 0.0)
    assert np.abs(b).max() > 0.0
