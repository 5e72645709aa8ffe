"""Pins of the oracle's velocity-pressure system (oracle.saddle: Eq. weakNavierStokes with the Q1 pressure) against
closed forms.  CPU only."""
import numpy as np
import pytest

import closed_forms
import workloads
from oracle import fe, momentum, physics, saddle, step

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def q1_z(n):
    r = np.arange(n + 1) / n
    Z, _, _ = np.meshgrid(r, r, r, indexing="ij")
    return Z.ravel()


def problem(n, p, phi, mdot, seed=1, **over):
    wl = workloads.random_workload(n, p, seed, geom="sphere", dirichlet_faces=0x1F, **over)
    wl.phi = phi
    wl.mdot = mdot
    return momentum.Problem.from_workload(wl)


@pytest.mark.parametrize("p", [2, 3])
def test_hydrostatic_pressure_is_exact(p):
    """Liquid at rest under gravity, walls on five faces, the top face z = 1 open (zero traction): the exact solution
    of the discrete system is x = 0, p = rho_l g_z (z - 1) (linear, so in the Q1 space; every integrand is integrated
    exactly), whatever the linearization velocity u0.  A sign or transposition mistake in the pressure term, or a
    pressure level not fixed by the open face, moves p."""
    n = 4
    N1 = (n + 1) ** 3
    pb = problem(n, p, np.ones(N1), np.zeros(N1))
    gz = -9.81
    f = saddle.body_force_load(pb, (0.0, 0.0, gz))
    x, pr = saddle.solve(pb, f)
    p_exact = pb.params["rho_l"] * gz * (q1_z(n) - 1.0)
    assert np.abs(x).max() < 1e-10 * np.abs(p_exact).max() * pb.mesh.h
    # the direct solve of the scaled saddle system (c_m rho ~ 1e7 against O(h^2) pressure couplings) rounds at ~1e-9
    assert np.abs(pr - p_exact).max() < 1e-8 * np.abs(p_exact).max()


def test_prescribed_pressure_gradient_is_recovered():
    """f = -B^T p*, g = 0 (no evaporation): K [0; p*] = [f; 0], and K is nonsingular with an open face, so the solve
    returns x = 0 and p = p* at every node (also on the open face)."""
    n = 4
    N1 = (n + 1) ** 3
    rng = np.random.default_rng(4)
    z = q1_z(n)
    pb = problem(n, 2, np.tanh((0.55 - z) / (2 * 0.25)), np.zeros(N1))
    B, _ = momentum.divergence(pb)
    pstar = rng.uniform(-1, 1, N1)
    x, pr = saddle.solve(pb, -(B.T @ pstar))
    assert np.abs(x).max() < 1e-9
    assert np.abs(pr - pstar).max() < 1e-8


def test_evaporating_slab_outflow_is_the_dilation_integral():
    """Flat evaporating interface z = 1/2 (liquid below) with a constant mdot, walls on five faces, top open, no
    force: the continuity row makes the outflow through the top face equal sum_j g_j = int v_dil exactly (the face
    integral of x . n is computed by face quadrature, independently of B), and int v_dil = mdot (1/rho_g - 1/rho_l)
    times the area (the gas velocity of App. A, Eq. stefan_diffuse_velocity, with the liquid at rest), up to the
    quadrature of the delta profile (within 2 %): evaporation expands the volume, the gas leaves through the open
    face."""
    n = 8
    N1 = (n + 1) ** 3
    z = q1_z(n)
    eps = 1.0 / n
    mdot = 0.5
    pb = problem(n, 2, np.tanh((0.5 - z) / (2 * eps)), np.full(N1, mdot))
    x, _ = saddle.solve(pb, np.zeros(3 * pb.mesh.n_u))
    out = saddle.top_outflow(pb.mesh, x)
    g = saddle.continuity_rhs(pb)
    assert out == pytest.approx(g.sum(), rel=1e-9)
    prm = pb.params
    closed = mdot * (1.0 / prm["rho_g"] - 1.0 / prm["rho_l"])
    assert closed > 0.0
    assert out == pytest.approx(closed, rel=0.02)


def test_closed_box_is_rejected():
    n = 3
    N1 = (n + 1) ** 3
    pb = problem(n, 2, np.ones(N1), np.zeros(N1))
    pb.params["dirichlet_faces"] = 0x3F
    with pytest.raises(ValueError):
        saddle.solve(pb, np.zeros(3 * pb.mesh.n_u))


# ---------------------------------------------------------------------------- 1D phase change (App. A), stationary
STEFAN = dict(eps=0.125, mdot=0.01, rho_l=1.0, rho_g=1e-3, mu=1e-3, z0=0.5)  # the parameters of Sec. 3.1, eps fixed


def stefan_case(n, dt=1.0, stress=1, **over):
    """Flat interface z = z0 (liquid below), inflow u_bar = mdot / rho_l through the bottom face (static interface),
    the top face open (zero pressure outlet), the four side faces Dirichlet with the exact 1D velocity, so that the 3D
    box holds the 1D solution.  Returns the mesh, the parameters, phi (Q1), the exact velocity u (Q_2, the Dirichlet
    data and the linearization velocity), mdot and the exact pressure at the Q1 nodes."""
    c = dict(STEFAN, **over)
    mesh = fe.Mesh(n, 2, 1.0)
    prm = workloads.default_params(n, 1.0, rho_l=c["rho_l"], rho_g=c["rho_g"], mu_l=c["mu"], mu_g=c["mu"],
                                   dirichlet_faces=0x1F, dt=dt, newton=0, variant=2, stress=stress)
    prm["eps"] = c["eps"]
    prm["c_mass"] = 1.0 / dt
    prm["dtau"] = min(c["eps"], dt)
    z1 = workloads.node_coords(n, 1)[:, 2]
    zu = workloads.node_coords(n, 2)[:, 2]
    phi = np.tanh((c["z0"] - z1) / (2 * c["eps"]))
    uz, _ = closed_forms.stefan_diffuse(c["z0"] - zu, c["eps"], c["mdot"], c["rho_l"], c["rho_g"])
    u = np.zeros(3 * mesh.n_u)
    u[2 * mesh.n_u:] = uz
    _, pex = closed_forms.stefan_diffuse(c["z0"] - z1, c["eps"], c["mdot"], c["rho_l"], c["rho_g"])
    jump = c["mdot"] * (1.0 / c["rho_g"] - 1.0 / c["rho_l"])
    return mesh, prm, phi, u, np.full(mesh.n_phi, c["mdot"]), pex, jump


def stefan_errors(n, stress=1):
    """One BDF1 Navier-Stokes step (dt = 1, quasi-steady) from the exact state: max nodal errors of the velocity and
    the pressure relative to the velocity jump and to the pressure jump mdot^2 (1/rho_g - 1/rho_l)."""
    mesh, prm, phi, u, md, pex, jump = stefan_case(n, stress=stress)
    pb = momentum.Problem(mesh=mesh, params=prm, phi=phi, u0=u, mdot=md)
    f = step.mass_load(pb, u)
    mask = pb.constrained()
    f[mask] = u[mask]  # Dirichlet data: inflow at the bottom, the exact profile on the side faces
    x, p = saddle.solve(pb, f)
    assert np.abs(x[mask] - u[mask]).max() == 0.0
    dp = STEFAN["mdot"] * jump
    return np.abs(x - u).max() / jump, np.abs(p - pex).max() / dp, p, x


def test_stationary_1d_phase_change_matches_the_diffuse_closed_form():
    """App. A: with the inflow u_bar = mdot / rho_l the interface is static and the diffuse model's velocity and
    pressure are Eqs. (stefan_diffuse_velocity), (stefan_diffuse_pressure).  The discrete step reproduces both with an
    error that shrinks under refinement at fixed eps (6^3 -> 8^3 cells: 5.5 % -> 2.1 % of the velocity jump, 15 % ->
    8.6 % of the pressure jump; a reversed dilation sign, a dropped source or an arithmetic density give errors of the
    order of the jumps or larger); the flow stays one-dimensional up to the same discretization error."""
    eu6, ep6, _, _ = stefan_errors(6)
    eu8, ep8, p8, x8 = stefan_errors(8)
    assert eu8 < 0.03 and ep8 < 0.1
    assert eu8 < eu6 / 2.0 and ep8 < ep6 / 1.5
    n_u = fe.Mesh(8, 2, 1.0).n_u
    assert np.abs(x8[:2 * n_u]).max() < 0.03 * STEFAN["mdot"] * (1.0 / STEFAN["rho_g"] - 1.0 / STEFAN["rho_l"])


def test_standard_stokes_shows_the_artificial_pressure_peak():
    """Sec. 3.1.2: with the uncorrected rate of deformation (standard Stokes) the evaporation-induced volumetric strain
    rate enters the viscous stress and the pressure in the interface zone rises above the liquid's (a peak of ~20 % of
    the jump on the centre line at 8^3, error > 40 %), which the corrected stress of Eq. (modified_viscous_stress)
    removes (the previous test)."""
    _, ep, p, _ = stefan_errors(8, stress=0)
    assert ep > 0.4
    n = 8
    dp = STEFAN["mdot"] ** 2 * (1.0 / STEFAN["rho_g"] - 1.0 / STEFAN["rho_l"])
    centre = p.reshape(n + 1, n + 1, n + 1)[:, n // 2, n // 2] / dp
    assert centre.max() > 1.15
