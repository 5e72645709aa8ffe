"""GPU parity of the velocity-pressure system (Eq. weakNavierStokes with the Q1 pressure) against oracle.saddle,
through the C ABI.

Tolerances: the apply evaluates the same Gauss sums as the oracle's assembled matrices (1e-12 relative).  The solve
stops at a relative residual of 1e-12; the saddle system couples O(rho c_m h^3) velocity rows with O(h^2) pressure
couplings (condition ~1e8 on these meshes), and the oracle's own direct solve rounds at ~1e-9 relative in the
pressure (its hydrostatic pin), so the solution bars are 1e-7 (velocity) and 1e-6 (pressure) relative in l2."""
import numpy as np
import pytest
import torch

import workloads
from oracle import fe, momentum, saddle

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    import paper_2401_07805_gb300 as evap
    from paper_2401_07805_gb300 import build
    if not os.path.exists(evap.library_path()):
        build.build()
    evap.lib()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make(wl):
    from paper_2401_07805_gb300 import Operator
    op = Operator(wl.n, wl.p, wl.L, dict(wl.params))
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    return op, momentum.Problem.from_workload(wl)


def q1_z(n):
    r = np.arange(n + 1) / n
    Z, _, _ = np.meshgrid(r, r, r, indexing="ij")
    return Z.ravel()


@pytest.mark.parametrize("n,p,faces,geom,seed", [(8, 2, 0x1F, "sphere", 2), (7, 2, 0x2B, "spheres", 5),
                                                 (5, 3, 0x1F, "sphere", 3), (6, 2, 0x3F, "deformed", 7)],
                         ids=["q2_open_top", "q2_ragged_mixed_faces", "q3_open_top", "q2_closed"])
def test_saddle_apply_against_oracle(n, p, faces, geom, seed):
    wl = workloads.random_workload(n, p, seed, geom=geom, dirichlet_faces=faces)
    op, pb = make(wl)
    rng = np.random.default_rng(seed + 10)
    x = rng.uniform(-1, 1, 3 * op.n_u)
    pr = rng.uniform(-1, 1, op.n_phi) * 1e3  # pressures of the size the inertia rows produce
    y, yp = op.apply_saddle(cuda(x), cuda(pr))
    ry, ryp = saddle.apply(pb, x, pr)
    assert rel(host(y), ry) < 1e-12
    assert rel(host(yp), ryp) < 1e-12
    # the pressure term alone (x = 0): -B^T p on the free rows, 0 on the constrained ones
    y0, yp0 = op.apply_saddle(cuda(np.zeros_like(x)), cuda(pr))
    B, _ = momentum.divergence(pb)
    assert rel(host(y0), -(B.T @ pr)) < 1e-12
    # B 0 = 0 up to the rounding of (B x - g) + g: the divergence row's source and g are summed in different orders
    assert np.abs(host(yp0)).max() < 1e-14 * max(np.abs(saddle.continuity_rhs(pb)).max(), 1e-300) + 1e-300


@pytest.mark.parametrize("n,p,seed", [(6, 2, 4), (4, 3, 6)], ids=["q2", "q3"])
def test_saddle_solve_against_oracle(n, p, seed):
    """Random right-hand side, evaporating sphere (mdot ~ U[0.5, 1.5]), walls on five faces, top open."""
    wl = workloads.random_workload(n, p, seed, geom="sphere", dirichlet_faces=0x1F)
    op, pb = make(wl)
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1, 1, 3 * op.n_u)
    f[pb.constrained()] = 0.0
    x, pr, info = op.solve_saddle(cuda(f), rtol=1e-12, max_iter=2000)
    xr, prr = saddle.solve(pb, f)
    assert info["converged"], info
    assert rel(host(x), xr) < 1e-7
    assert rel(host(pr), prr) < 1e-6


def test_saddle_solve_hydrostatic():
    """Liquid at rest under gravity with the top open: x = 0 and p = rho_l g_z (z - 1) (the oracle's pin)."""
    n = 8
    N1 = (n + 1) ** 3
    wl = workloads.random_workload(n, 2, 1, geom="sphere", dirichlet_faces=0x1F)
    wl.phi = np.ones(N1)
    wl.mdot = np.zeros(N1)
    op, pb = make(wl)
    gz = -9.81
    f = saddle.body_force_load(pb, (0.0, 0.0, gz))
    x, pr, info = op.solve_saddle(cuda(f), rtol=1e-12, max_iter=2000)
    p_exact = pb.params["rho_l"] * gz * (q1_z(n) - 1.0)
    assert info["converged"], info
    assert np.abs(host(pr) - p_exact).max() < 1e-7 * np.abs(p_exact).max()
    assert np.abs(host(x)).max() < 1e-7


def test_saddle_solve_evaporating_slab_outflow():
    """Flat evaporating interface, top open, no force: the outflow through the top face equals sum_j g_j (the
    continuity row, to the solve tolerance) and mdot (1/rho_g - 1/rho_l) > 0 per unit area within 2 % (the gas
    leaves: App. A)."""
    n = 8
    N1 = (n + 1) ** 3
    wl = workloads.random_workload(n, 2, 1, geom="sphere", dirichlet_faces=0x1F)
    wl.phi = np.tanh((0.5 - q1_z(n)) / (2.0 / n))
    mdot = 0.5
    wl.mdot = np.full(N1, mdot)
    op, pb = make(wl)
    # |[f; g]| = |g| is small against the rounding of the inertia rows (rho c_m h^3 |x|): the double-float apply rounds
    # at ~4e-15 of their scale, which puts the attainable relative residual near 2e-10 here; 1e-9 is reachable
    x, _, info = op.solve_saddle(cuda(np.zeros(3 * op.n_u)), rtol=1e-9, max_iter=2000)
    assert info["converged"], info
    out = saddle.top_outflow(pb.mesh, host(x))
    g = saddle.continuity_rhs(pb)
    assert out == pytest.approx(g.sum(), rel=1e-6)
    prm = pb.params
    closed = mdot * (1.0 / prm["rho_g"] - 1.0 / prm["rho_l"])
    assert closed > 0.0
    assert out == pytest.approx(closed, rel=0.02)


def test_saddle_solve_dirichlet_data_against_oracle():
    """Non-homogeneous Dirichlet data (the 1D phase change of App. A: inflow through the bottom face, the exact
    profile on the side faces) lifted into the free rows, against the oracle's direct solve of the same system K_D;
    the Dirichlet entries of the solution are the data exactly."""
    from oracle import step
    from test_oracle_saddle import stefan_case
    n = 6
    mesh, prm, phi, u, md, _, _ = stefan_case(n)
    from paper_2401_07805_gb300 import Operator
    op = Operator(n, 2, 1.0, dict(prm))
    op.set_fields(cuda(phi), cuda(u), cuda(md))
    pb = momentum.Problem(mesh=mesh, params=prm, phi=phi, u0=u, mdot=md)
    f = step.mass_load(pb, u)
    mask = pb.constrained()
    f[mask] = u[mask]
    x, pr, info = op.solve_saddle(cuda(f), rtol=1e-12, max_iter=3000)
    assert info["converged"], info
    xr, prr = saddle.solve(pb, f)
    assert np.array_equal(host(x)[mask], u[mask])
    assert rel(host(x), xr) < 1e-7
    assert rel(host(pr), prr) < 1e-6


def test_saddle_solve_rejects_a_closed_box():
    from paper_2401_07805_gb300 import EvapError
    wl = workloads.random_workload(4, 2, 1, geom="sphere")
    op, _ = make(wl)
    with pytest.raises(EvapError):
        op.solve_saddle(cuda(np.zeros(3 * op.n_u)))


def test_input_checks_report_non_finite_entries():
    """With checks on, a NaN or Inf in an input array returns EVAP_ENONFINITE before any work (the output is left
    untouched); with checks off the same call runs.  The check covers set_fields, the applies and the solves."""
    from paper_2401_07805_gb300 import EvapError
    wl = workloads.random_workload(5, 2, 3, geom="sphere", dirichlet_faces=0x1F)
    op, _ = make(wl)
    x = np.random.default_rng(1).uniform(-1, 1, 3 * op.n_u)
    x[17] = np.nan
    op.set_checks(True)
    y = torch.full((3 * op.n_u,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(EvapError, match="ENONFINITE"):
        op.apply_momentum(cuda(x), prec=64, out=y)
    assert bool((y == 7.0).all())
    with pytest.raises(EvapError, match="ENONFINITE"):
        op.apply_momentum(cuda(x).float(), prec=32)
    f = np.zeros(3 * op.n_u)
    f[5] = np.inf
    with pytest.raises(EvapError, match="ENONFINITE"):
        op.solve_saddle(cuda(f))
    phi = wl.phi.copy()
    phi[3] = np.nan
    with pytest.raises(EvapError, match="ENONFINITE"):
        op.set_fields(cuda(phi), cuda(wl.u0), cuda(wl.mdot))
    x[17] = 0.0
    op.apply_momentum(cuda(x), prec=64, out=y)  # finite again: runs
    op.set_checks(False)
    x[17] = np.nan
    op.apply_momentum(cuda(x), prec=64, out=y)  # checks off: no error, NaN propagates
    assert bool(torch.isnan(y).any())
