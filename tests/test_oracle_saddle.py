"""Pins of the oracle's velocity-pressure system (oracle.saddle: Eq. weakNavierStokes with the Q1 pressure) against
closed forms.  CPU only."""
import numpy as np
import pytest

import workloads
from oracle import fe, momentum, physics, saddle

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
    integral of x . n is computed by face quadrature, independently of B), and int v_dil = mdot (1/rho_l - 1/rho_g)
    times the area, up to the quadrature of the delta profile (within 2 %)."""
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
    closed = mdot * (1.0 / prm["rho_l"] - 1.0 / prm["rho_g"])
    assert out == pytest.approx(closed, rel=0.02)


def test_closed_box_is_rejected():
    n = 3
    N1 = (n + 1) ** 3
    pb = problem(n, 2, np.ones(N1), np.zeros(N1))
    pb.params["dirichlet_faces"] = 0x3F
    with pytest.raises(ValueError):
        saddle.solve(pb, np.zeros(3 * pb.mesh.n_u))
