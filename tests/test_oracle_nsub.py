"""Pins of the oracle's subdivided level-set mesh (Sec. 2.5: the level set on the Navier-Stokes mesh subdivided
n_sub = 2 times per direction, Q1 on each sub-cell; the pressure stays Q1 on the Navier-Stokes mesh).  CPU only.

The central pin: a level set (and mass flux) that is trilinear on every velocity cell is reproduced exactly by the
subdivided space (a trilinear function is trilinear on each sub-cell), so with the fine nodal values taken from the
coarse Q1 field every operator of the subdivided discretization must equal the n_sub = 1 operator up to rounding,
and the gradients with respect to the fine nodal values must restrict (by the transpose of that interpolation) to
the n_sub = 1 gradients.  A wrong sub-cell, a wrong gradient scale 1/(h/2), or a node-order mistake breaks it."""
import numpy as np
import pytest

import workloads
from oracle import adjoint, fe, levelset, momentum, physics, transport

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def prolongation(n):
    """P [(2n+1)^3, (n+1)^3]: the coarse Q1 interpolant at the fine Q1 nodes (1D weights 1, 1/2)."""
    import scipy.sparse as sp
    rows, cols, vals = [], [], []
    for i in range(2 * n + 1):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [i // 2, i // 2 + 1]; vals += [0.5, 0.5]
    P1 = sp.csr_matrix((vals, (rows, cols)), shape=(2 * n + 1, n + 1))
    return sp.kron(sp.kron(P1, P1), P1).tocsr()   # z slowest, x fastest


def test_iso_q1_basis():
    """Partition of unity, exact gradients of linear fields at every point (also on the sub-cell faces), and the
    sub-cell rule at t = 1/2 (the upper sub-cell's slopes)."""
    t = np.array([0.0, 0.1127, 0.25, 0.5, 0.8873, 1.0])
    V, D = fe.iso_q1_1d(t, 2)
    np.testing.assert_allclose(V.sum(0), 1.0, atol=1e-15)
    np.testing.assert_allclose(D.sum(0), 0.0, atol=1e-15)
    xs = np.array([0.0, 0.5, 1.0])
    np.testing.assert_allclose(xs @ V, t, atol=1e-15)
    np.testing.assert_allclose(xs @ D, 1.0, atol=1e-15)
    np.testing.assert_array_equal(D[:, 3], [0.0, -2.0, 2.0])
    V1, D1 = fe.iso_q1_1d(t, 1)
    np.testing.assert_allclose(V1, np.stack([1 - t, t]), atol=1e-15)


@pytest.mark.parametrize("p,stress,zone,newton", [(2, 1, 0, 1), (3, 1, 1, 0), (2, 0, 0, 1)])
def test_subdivided_operator_reproduces_coarse_level_set(p, stress, zone, newton):
    """Momentum apply, divergence row and adjoint with the fine level set = the coarse Q1 field at the fine nodes equal
    the n_sub = 1 operator; the fine gradients of phi and mdot restrict to the coarse ones (P^T g_fine = g_coarse)."""
    n = 3
    wl = workloads.random_workload(n, p=p, seed=4, geom="sphere", dirichlet_faces=0x15, stress=stress,
                                   corr_zone=zone, newton=newton)
    wl.params["eps"] = 0.3
    pb1 = momentum.Problem.from_workload(wl)
    P = prolongation(n)
    pb2 = momentum.Problem(mesh=fe.Mesh(n, p, 1.0, 2), params=dict(wl.params, n_sub=2), phi=P @ wl.phi,
                           u0=wl.u0.copy(), mdot=P @ wl.mdot)
    y1, yp1 = momentum.apply(pb1, wl.x, with_divergence=True)
    y2, yp2 = momentum.apply(pb2, wl.x, with_divergence=True)
    np.testing.assert_allclose(y2, y1, rtol=1e-12, atol=1e-12 * np.abs(y1).max())
    np.testing.assert_allclose(yp2, yp1, rtol=1e-12, atol=1e-12 * np.abs(yp1).max())
    rng = np.random.default_rng(1)
    w = rng.uniform(-1, 1, wl.x.shape)
    wp = rng.uniform(-1, 1, pb1.mesh.n_p)
    gu1, gphi1, gm1 = adjoint.param_gradients(pb1, wl.x, w, wp)
    gu2, gphi2, gm2 = adjoint.param_gradients(pb2, wl.x, w, wp)
    assert gphi2.shape == (pb2.mesh.n_phi,) and gm2.shape == (pb2.mesh.n_phi,)
    np.testing.assert_allclose(gu2, gu1, rtol=1e-12, atol=1e-12 * np.abs(gu1).max())
    np.testing.assert_allclose(P.T @ gphi2, gphi1, rtol=1e-10, atol=1e-11 * np.abs(gphi1).max())
    np.testing.assert_allclose(P.T @ gm2, gm1, rtol=1e-10, atol=1e-11 * np.abs(gm1).max())


def test_subdivided_adjoint_matches_central_differences():
    """Fine-space gradients of L = w.A x + w_p.(B x - g) against central differences in random fine-node directions
    of phi (h = 1e-6) and mdot (L is linear in mdot)."""
    n = 2
    wl = workloads.random_workload(n, seed=7, geom="sphere", dirichlet_faces=0, n_sub=2)
    wl.params["eps"] = 0.35
    rng = np.random.default_rng(5)
    wl.phi = rng.uniform(-0.9, 0.9, wl.phi.shape)
    pb = momentum.Problem.from_workload(wl)
    assert pb.mesh.n_sub == 2 and wl.phi.size == pb.mesh.n_phi == 125
    w = rng.uniform(-1, 1, wl.x.shape)
    wp = rng.uniform(-1, 1, pb.mesh.n_p)
    _, gphi, gm = adjoint.param_gradients(pb, wl.x, w, wp)
    for _ in range(4):
        dphi = rng.uniform(-1, 1, wl.phi.shape)
        hh = 1e-6
        lp = adjoint.loss(momentum.Problem(mesh=pb.mesh, params=pb.params, phi=wl.phi + hh * dphi, u0=wl.u0,
                                           mdot=wl.mdot), wl.x, w, wp)
        lm = adjoint.loss(momentum.Problem(mesh=pb.mesh, params=pb.params, phi=wl.phi - hh * dphi, u0=wl.u0,
                                           mdot=wl.mdot), wl.x, w, wp)
        assert (lp - lm) / (2 * hh) == pytest.approx(gphi @ dphi, rel=1e-5, abs=1e-9)
        dm = rng.uniform(-1, 1, wl.phi.shape)
        lp = adjoint.loss(momentum.Problem(mesh=pb.mesh, params=pb.params, phi=wl.phi, u0=wl.u0, mdot=wl.mdot + dm),
                          wl.x, w, wp)
        lm = adjoint.loss(momentum.Problem(mesh=pb.mesh, params=pb.params, phi=wl.phi, u0=wl.u0, mdot=wl.mdot - dm),
                          wl.x, w, wp)
        assert (lp - lm) / 2 == pytest.approx(gm @ dm, rel=1e-9, abs=1e-12)


def test_subdivided_level_set_operators_live_on_the_fine_mesh():
    """The level-set operators of the subdivided discretization are the Q1 operators of the fine mesh: exact mass
    of the unit field (1^T M 1 = 1), zero advection of a constant field and zero reinitialization stiffness on it."""
    n = 3
    mesh1 = fe.Mesh(2 * n, 1, 1.0)
    N = mesh1.n_phi
    one = np.ones(N)
    rng = np.random.default_rng(2)
    phi = rng.uniform(-1, 1, N)
    ug = rng.uniform(-1, 1, 3 * N)
    prm = workloads.default_params(n, 1.0)
    y = levelset.apply(mesh1, "advect", one, phi, ug, prm)
    assert one @ y == pytest.approx(1.0, rel=1e-13)  # 1^T (M + theta dt C(u)) 1 = |Omega| + theta dt int u.grad 1
    yr = levelset.apply(mesh1, "reinit", one, phi, ug, prm)
    assert one @ yr == pytest.approx(1.0 / prm["dtau"], rel=1e-13)


@pytest.mark.parametrize("variant", [1, 2])
def test_subdivided_transport_velocity_on_the_static_flat_interface(variant):
    """Variant 1 (Eq. transport_vel_local_continuous) vanishes at every fine node of the static flat interface
    (u = mdot / rho(phi) e_z from the fine level set, App. A with u_bar = mdot / rho_l); variant 2 vanishes up to the
    interpolation error of u at the projected point (< 1e-3 of the velocity jump)."""
    eps = 0.1
    errs = []
    for n in (4, 8):
        mesh = fe.Mesh(n, 2, 1.0, 2)
        prm = workloads.default_params(n, eps=eps, variant=variant, rho_l=1.0, rho_g=0.5, n_sub=2)
        zf = workloads.node_coords(2 * n, 1)[:, 2]
        phi = np.tanh((0.5 - zf) / (2 * eps))
        zq = workloads.node_coords(n, 2)[:, 2]
        u0 = np.zeros(3 * mesh.n_u)
        u0[2 * mesh.n_u:] = 1.0 / physics.density(physics.heaviside(np.tanh((0.5 - zq) / (2 * eps)), eps), 1.0, 0.5)
        ug, flags = transport.transport_velocity(mesh, phi, u0, np.ones(mesh.n_phi), prm)
        assert ug.shape == (3, mesh.n_phi) and flags.sum() == 0
        np.testing.assert_allclose(ug[:2], 0.0, atol=1e-14)
        errs.append(np.abs(ug[2]).max())
    if variant == 1:
        assert max(errs) < 1e-14
    else:
        assert errs[1] < 1e-3 * (1.0 / 0.5 - 1.0) and errs[1] < errs[0]
