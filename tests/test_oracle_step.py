"""Pins of the oracle's coupled time step (oracle.step: BDF1 Picard Navier-Stokes step, then Algorithm 2) against
closed forms.  CPU only."""
import numpy as np
import pytest

import workloads
from oracle import fe, step

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def slab_case(n, mdot_val, z0=0.55):
    z = workloads.node_coords(n, 1)[:, 2]
    prm = workloads.default_params(n, 1.0, ratio=10.0, dirichlet_faces=0x1F, dt=0.02, newton=0, variant=2)
    prm["c_mass"] = 1.0 / prm["dt"]
    prm["dtau"] = min(prm["eps"], prm["dt"])
    phi = np.tanh((z0 - z) / (2 * prm["eps"]))
    mesh = fe.Mesh(n, 2, 1.0)
    return mesh, prm, phi, np.full(mesh.n_phi, float(mdot_val))


def interface_height(phi, n):
    """z of phi = 0 on the vertical line through the domain centre (linear interpolation between nodes)."""
    m = n + 1
    col = phi.reshape(m, m, m)[:, m // 2, m // 2]
    zz = np.arange(m) / n
    for k in range(m - 1):
        if col[k] > 0 >= col[k + 1]:
            return zz[k] + col[k] / (col[k] - col[k + 1]) * (zz[k + 1] - zz[k])
    raise AssertionError("no interface on the centre line")


def test_evaporating_slab_recedes_at_mdot_over_rho_l():
    """Liquid at rest below a flat interface (walls on five faces, the top open), constant mdot: the liquid end of
    the interface region does not move, so the variant-2 transport velocity is mdot / rho_l n and the interface
    recedes into the liquid at mdot / rho_l (the sharp solution of the 1D phase-change problem with no inflow,
    App. evapor_stefan).  Over three steps the displacement matches to 3 %; a dropped or sign-flipped evaporation
    term gives 0 or -100 %."""
    n = 8  # eps = h: the interface zone |d| < 3 eps stays one cell away from the bottom wall and the top face
    mesh, prm, phi, mdot = slab_case(n, 50.0, z0=0.5)
    u = np.zeros(3 * mesh.n_u)
    p = np.zeros(mesh.n_phi)
    z0 = interface_height(phi, n)
    for k in range(3):
        phi, u, p = step.time_step(mesh, prm, phi, u, p, mdot, fp_iters=2, reinit_steps=2)
        moved = z0 - interface_height(phi, n)
        assert moved == pytest.approx((k + 1) * prm["dt"] * 50.0 / prm["rho_l"], rel=0.03)


def test_rest_state_without_evaporation_stays_at_rest():
    """No evaporation, no force, fluid at rest: f = 0 and g = 0, so the Navier-Stokes step returns exactly u = 0,
    p = 0; the level set then only feels the reinitialization of the discrete tanh profile (a few 1e-3)."""
    n = 6
    mesh, prm, phi, _ = slab_case(n, 0.0)
    ph, u, p = step.time_step(mesh, prm, phi, np.zeros(3 * mesh.n_u), np.zeros(mesh.n_phi), np.zeros(mesh.n_phi),
                              fp_iters=1, reinit_steps=1)
    assert np.abs(u).max() == 0.0 and np.abs(p).max() == 0.0
    assert np.abs(ph - phi).max() < 5e-3


def test_bdf2_steps_recede_at_the_same_rate():
    """One BDF1 step, then BDF2 steps with u^(n-1): the recession rate stays mdot / rho_l (3 %), and the BDF2 load
    (4 u^n - u^(n-1)) / 3 reduces to u^n for a steady velocity, so the rest state stays exactly at rest."""
    n = 8
    mesh, prm, phi, mdot = slab_case(n, 50.0, z0=0.5)
    u_prev = np.zeros(3 * mesh.n_u)
    u = np.zeros(3 * mesh.n_u)
    p = np.zeros(mesh.n_phi)
    z0 = interface_height(phi, n)
    phi, u1, p = step.time_step(mesh, prm, phi, u, p, mdot)
    for k in range(2):
        phi, u2, p = step.time_step(mesh, prm, phi, u1, p, mdot, u_prev=u)
        u, u1 = u1, u2
        moved = z0 - interface_height(phi, n)
        assert moved == pytest.approx((k + 2) * prm["dt"] * 50.0 / prm["rho_l"], rel=0.03)
    _, ur, pr = step.time_step(mesh, prm, np.tanh((0.5 - workloads.node_coords(n, 1)[:, 2]) / (2 * prm["eps"])),
                               np.zeros(3 * mesh.n_u), np.zeros(mesh.n_phi), np.zeros(mesh.n_phi),
                               u_prev=np.zeros(3 * mesh.n_u))
    assert np.abs(ur).max() == 0.0 and np.abs(pr).max() == 0.0


def test_newton_iterations_converge_quadratically():
    """App. D's Newton iterations on the strong-convection case of the Picard test: the nonlinear residual falls
    quadratically (|R^(k+1)| <= C |R^(k)|^2 with a C that holds over the iterations, far faster than the Picard
    iterations' geometric rate) and the converged step equals the converged Picard step (both solve the same
    nonlinear system)."""
    n = 5
    mesh, prm, phi, mdot = slab_case(n, 20.0)
    rng = np.random.default_rng(3)
    u = rng.uniform(-0.3, 0.3, 3 * mesh.n_u)
    from oracle import momentum
    pb = momentum.Problem(mesh=mesh, params=dict(prm), phi=phi, u0=u, mdot=mdot)
    u[pb.constrained()] = 0.0
    p = np.zeros(mesh.n_phi)
    res_n, res_p = [], []
    _, un, pn = step.time_step(mesh, dict(prm, newton=1), phi, u, p, mdot, fp_iters=1, reinit_steps=0, picard_iters=4,
                               residuals=res_n)
    _, up, pp = step.time_step(mesh, prm, phi, u, p, mdot, fp_iters=1, reinit_steps=0, picard_iters=12,
                               residuals=res_p)
    assert len(res_n) == 3
    # quadratic (observed 1.2 -> 5.8e-4 -> 9.5e-10): r_(k+1) <= 1e-2 r_k^2, while the Picard residuals fall by a
    # constant factor of ~0.05 per iteration
    for a, b in zip(res_n, res_n[1:]):
        assert b < 1e-2 * a * a
    assert res_n[2] < 1e-6 * res_p[2]
    np.testing.assert_allclose(un, up, rtol=0, atol=1e-8 * np.abs(up).max())
    np.testing.assert_allclose(pn, pp, rtol=0, atol=1e-6 * np.abs(pp).max())


def test_picard_iterations_contract_the_nonlinear_residual():
    """A strong convection (u^n = 0.3 in the gas, dt = 0.02, about 0.1 cells per step): the Picard iterations of a
    step contract the nonlinear residual |[f; g] - K(u^(k)) [u^(k); p^(k)]| geometrically, and a tolerance stops them
    early; one iteration leaves the semi-implicit step."""
    n = 5
    mesh, prm, phi, mdot = slab_case(n, 20.0)
    rng = np.random.default_rng(3)
    u = rng.uniform(-0.3, 0.3, 3 * mesh.n_u)
    from oracle import momentum
    pb = momentum.Problem(mesh=mesh, params=dict(prm), phi=phi, u0=u, mdot=mdot)
    u[pb.constrained()] = 0.0
    p = np.zeros(mesh.n_phi)
    res = []
    step.time_step(mesh, prm, phi, u, p, mdot, fp_iters=1, reinit_steps=0, picard_iters=5, residuals=res)
    assert len(res) == 4
    for a, b in zip(res, res[1:]):
        assert b < 0.2 * a
    res2 = []
    step.time_step(mesh, prm, phi, u, p, mdot, fp_iters=1, reinit_steps=0, picard_iters=5, picard_atol=res[1] * 1.01,
                   residuals=res2)
    assert len(res2) == 2


def test_uniform_translation_is_preserved():
    """No walls (every face open), two phases, no evaporation or force: a uniform velocity U is an exact solution of
    the Picard step (no convection, stress or pressure), so a BDF1 step and a BDF2 step (u^(n-1) = U) both return
    u = U and p = 0; an inertia load of the wrong size or BDF2 weights that do not sum to one move it.  The interface
    is carried with the transport velocity U (variant 1 without evaporation) by about U_z dt."""
    n = 4
    z = workloads.node_coords(n, 1)[:, 2]
    prm = workloads.default_params(n, 1.0, ratio=10.0, dirichlet_faces=0, dt=0.02, newton=0, variant=1)
    prm["c_mass"] = 1.0 / prm["dt"]
    prm["dtau"] = min(prm["eps"], prm["dt"])
    phi = np.tanh((0.55 - z) / (2 * prm["eps"]))
    mesh = fe.Mesh(n, 2, 1.0)
    U = np.array([0.2, -0.1, 0.5])
    u = np.repeat(U[:, None], mesh.n_u, axis=1).ravel()
    mdot = np.zeros(mesh.n_phi)
    for u_prev in (None, u):
        ph, u1, p1 = step.time_step(mesh, prm, phi, u, np.zeros(mesh.n_phi), mdot, fp_iters=1, reinit_steps=0,
                                    u_prev=u_prev)
        assert np.abs(u1 - u).max() < 1e-9 * np.abs(u).max()
        # p = 0 up to the rounding of the direct solve, relative to the inertia pressure scale rho_l c_m |U| h
        assert np.abs(p1).max() < 1e-11 * prm["rho_l"] * prm["c_mass"] * np.abs(U).max() * mesh.h
    assert interface_height(ph, n) - interface_height(phi, n) == pytest.approx(U[2] * prm["dt"], rel=0.05)


def test_stationary_1d_phase_change_step():
    """App. A through the whole step (Navier-Stokes step with two Picard iterations, then Algorithm 2): from the exact
    diffuse state with the static inflow u_bar = mdot / rho_l, the step returns the closed-form velocity and pressure
    (Eqs. stefan_diffuse_velocity, stefan_diffuse_pressure) within the discretization error of the 6^3 mesh, and the
    interface does not move (variant 2: u(x_l) + mdot / rho_l n = u_bar - mdot / rho_l = 0)."""
    from test_oracle_saddle import STEFAN, stefan_case
    n = 6
    mesh, prm, phi, u, md, pex, jump = stefan_case(n)
    ph1, u1, p1 = step.time_step(mesh, prm, phi, u, np.zeros(mesh.n_phi), md, fp_iters=2, reinit_steps=2,
                                 picard_iters=2)
    assert np.abs(u1 - u).max() < 0.06 * jump
    assert np.abs(p1 - pex).max() < 0.17 * STEFAN["mdot"] * jump
    assert abs(interface_height(ph1, n) - interface_height(phi, n)) < 0.01 * mesh.h
