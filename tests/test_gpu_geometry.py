"""GPU parity of the level-set geometry sub-solver (projected normal, curvature, reinitialization) against the
oracle's direct solves (oracle.geometry), through the C ABI.

Tolerances (relative l2): the CUDA path solves each system by CG to |r| <= 1e-12 |r_0|; the systems are well
conditioned (M + 2 h^2 K: condition number ~25; the reinitialization matrix M/dtau + eps K_n with dtau = eps = h:
~1 + 12 eps dtau / h^2 ~ 13), so the solution error is <= ~1e-11.  Bar: 1e-10 for one solve; 1e-9 after several
reinitialization steps.  Single operator applies with the nodal normal: 1e-12 (same Gauss sums)."""
import numpy as np
import pytest
import torch

import workloads
from oracle import fe, geometry

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
    a = host(a) if isinstance(a, torch.Tensor) else a
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make_op(wl):
    from paper_2401_07805_gb300 import Operator
    op = Operator(wl.n, wl.p, wl.L, dict(wl.params))
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    return op


CASES = [("sphere8", {}), ("ragged7", dict(n=7, geom="sphere", seed=4)), ("spheres9", dict(n=9, geom="spheres", seed=6)),
         ("deformed10", dict(n=10, geom="deformed", seed=5))]


def workload(name, kw):
    if not kw:
        return workloads.make_workload(name)
    return workloads.random_workload(kw["n"], 2, kw["seed"], geom=kw["geom"])


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_projected_normal_and_curvature(name, kw):
    wl = workload(name, kw)
    op = make_op(wl)
    mesh = fe.Mesh(wl.n, 1, wl.L)
    n, info = op.projected_normal()
    assert info["converged"] and info["relres"] <= 1e-12
    n_ref = geometry.projected_normal(mesh, wl.phi, wl.params["eta_n"])
    assert rel(n, n_ref.ravel()) < 1e-10
    # curvature of the same (oracle) normal field on both sides
    kappa, kinfo = op.curvature(cuda(n_ref.ravel()))
    assert kinfo["converged"]
    k_ref = geometry.curvature(mesh, n_ref, wl.params["eta_kappa"])
    assert rel(kappa, k_ref) < 1e-10


@pytest.mark.parametrize("nodal", [False, True], ids=["unit_normal", "projected_normal"])
def test_reinitialization_steps(nodal):
    wl = workloads.random_workload(8, 2, 11, geom="sphere")
    op = make_op(wl)
    mesh = fe.Mesh(wl.n, 1, wl.L)
    eps, dtau = wl.params["eps"], wl.params["dtau"]
    nf = geometry.projected_normal(mesh, wl.phi) if nodal else None
    if nodal:
        op.set_levelset_normal(cuda(nf.ravel()))
    # a perturbed profile so that the steps move it
    psi0 = np.tanh(np.arctanh(np.clip(wl.phi, -0.999999, 0.999999)) * 0.6)
    psi, info = op.reinitialize(cuda(psi0), 3)
    ref, change = geometry.reinitialize(mesh, wl.phi, nf, eps, dtau, 3, psi0=psi0)
    assert info["converged"]
    assert rel(psi, ref) < 1e-9
    assert info["last_change"] == pytest.approx(change, rel=1e-6)
    # the operators with the nodal normal, one apply each
    x = np.random.default_rng(2).uniform(-1, 1, mesh.n_phi)
    y = op.apply_levelset(cuda(x), mode="reinit")
    assert rel(y, geometry.reinit_matrix(mesh, wl.phi, nf, eps, dtau) @ x) < 1e-12
    r = op.apply_levelset(cuda(x), mode="reinit_rhs")
    assert rel(r, geometry.reinit_rhs(mesh, wl.phi, nf, x, dtau)) < 1e-12
    op.set_levelset_normal(None)
    y0 = op.apply_levelset(cuda(x), mode="reinit")
    assert rel(y0, geometry.reinit_matrix(mesh, wl.phi, None, eps, dtau) @ x) < 1e-12


def test_reinitialize_zero_steps_and_arguments():
    from paper_2401_07805_gb300 import EvapError
    wl = workloads.make_workload("sphere8")
    op = make_op(wl)
    psi, info = op.reinitialize(cuda(wl.phi), 0)
    assert np.array_equal(host(psi), wl.phi) and info["iters"] == 0 and info["last_change"] == 0.0
    with pytest.raises(EvapError):
        op.reinitialize(cuda(wl.phi), -1)


def test_full_size_geometry_properties():
    """48^3 sphere (R = 0.25): the curvature at the interface nodes is 2/R within the discretization error, the
    reinitialization conserves int psi to rounding, and every CG solve converges."""
    wl = workloads.make_workload("sphere48")
    op = make_op(wl)
    mesh = fe.Mesh(wl.n, 1, wl.L)
    n, info = op.projected_normal()
    assert info["converged"]
    kappa, kinfo = op.curvature(n)
    assert kinfo["converged"]
    r1 = np.arange(mesh.n + 1) * mesh.h
    Z, Y, X = np.meshgrid(r1, r1, r1, indexing="ij")
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2).ravel()
    band = np.abs(r - 0.25) < 0.5 * mesh.h
    assert np.median(host(kappa)[band]) == pytest.approx(2.0 / 0.25, rel=0.05)
    op.set_levelset_normal(n)
    psi, rinfo = op.reinitialize(cuda(wl.phi), 5)
    assert rinfo["converged"]
    M = geometry.helmholtz_matrix(mesh, 0.0)
    one = np.ones(mesh.n_phi)
    m0, m1 = one @ (M @ wl.phi), one @ (M @ host(psi))
    assert abs(m1 - m0) < 1e-11 * abs(m0)


# ------------------------------------------------------------------------------------ advection (step 1)
def _q1_xyz(n):
    r = np.arange(n + 1) / n
    Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def test_advection_of_a_linear_field_is_exact():
    """phi = a . x + b, uniform velocity U, variant 1 without evaporation: phi^(n+1) = phi^n - dt U . a exactly
    (up to the GMRES tolerance |r| <= 1e-12 |b| of the step, about 1e-11 of max |phi| in the solution), and the
    second pass (the same system: u_Gamma does not depend on phi) changes nothing beyond that."""
    n = 9
    wl = workloads.random_workload(n, 2, 1, geom="sphere", variant=1, dt=0.01)
    U = np.array([0.3, -0.2, 0.5])
    wl.u0 = np.repeat(U[:, None], (2 * n + 1) ** 3, axis=1).ravel()
    wl.mdot = np.zeros((n + 1) ** 3)
    x, y, z = _q1_xyz(n)
    a = np.array([0.1, 0.05, -0.08])
    wl.phi = a[0] * x + a[1] * y + a[2] * z + 0.01
    op = make_op(wl)
    phi, info = op.advect_levelset(2)
    shift = wl.params["dt"] * float(U @ a)
    assert info["converged"] and info["fp_iters"] == 2
    assert np.abs(host(phi) - (wl.phi - shift)).max() < 1e-11
    assert info["last_change"] < 1e-11 * np.sqrt(wl.phi.size)


@pytest.mark.parametrize("n,geom,seed", [(8, "sphere", 3), (7, "spheres", 4)], ids=["sphere8", "ragged7"])
def test_advection_fixed_point_variant1_against_oracle(n, geom, seed):
    """Variant 1 (u_Gamma = u + mdot / rho(phi) n(phi) at the node: no iteration, GPU and oracle agree to 1e-13):
    three fixed-point passes with dt = 0.01 (about 0.1 cells per step), element by element against the oracle's
    direct solves.  Each GMRES solve stops at |r| <= 1e-12 |b| (b ~ M phi^n; the Jacobi-scaled operator is
    mass-dominated, condition ~10), an error of about 1e-11 of |phi^n|: bar 1e-10 |phi^n| on phi^(n+1), and 1e-7
    relative on the increment phi^(n+1) - phi^n (1 to 5 % of |phi^n|); the last change (a difference of two
    solutions) to 1e-3."""
    wl = workloads.random_workload(n, 2, seed, geom=geom, variant=1, dt=0.01)
    op = make_op(wl)
    phi, info = op.advect_levelset(3)
    mesh_u = fe.Mesh(n, 2, 1.0)
    ref, changes = geometry.advect_levelset(mesh_u, wl.phi, wl.u0, wl.mdot, wl.params, 3)
    assert info["converged"] and info["fp_iters"] == 3
    assert np.linalg.norm(host(phi) - ref) < 1e-10 * np.linalg.norm(wl.phi)
    assert rel(host(phi) - wl.phi, ref - wl.phi) < 1e-7
    assert info["last_change"] == pytest.approx(changes[-1], rel=1e-3, abs=1e-9)


def test_advection_fixed_point_variant2_against_oracle():
    """Variant 2 (closest points on the liquid-side isocontour, eps = h/2 so that it exists inside the drop; smooth
    velocity): the closest-point iteration resolves u_Gamma only to its stopping resolution and may end on another
    local minimum at a crease node, so the passes are checked one by one.  For K = 1, 2: the transport velocity of
    pass K (left on the mesh) is the oracle's u_Gamma of clamp(phi^(K-1)) at the transport-velocity bar (flags agree
    on >= 98 % of the nodes, >= 99 % of the nodes unflagged on both sides within 1e-6 of the velocity scale), and
    phi^(K) is the oracle's Crank-Nicolson step with that velocity (the solve bar of the variant-1 test: 1e-10
    |phi^n|, 1e-7 relative on the increment)."""
    from oracle import transport
    n = 8
    wl = workloads.random_workload(n, 2, 9, geom="sphere", variant=2, dt=0.01, eps=0.5 / n)
    X = workloads.node_coords(n, 2)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    wl.u0 = np.concatenate([0.5 * np.sin(2 * np.pi * y), 0.4 * np.cos(2 * np.pi * x),
                            0.3 * np.sin(2 * np.pi * (x + z))])
    wl.mdot = np.full((n + 1) ** 3, 300.0)
    op = make_op(wl)
    mesh_u, mesh1 = fe.Mesh(n, 2, 1.0), fe.Mesh(n, 1, 1.0)
    prev = np.clip(wl.phi, -1.0, 1.0)
    for K in (1, 2):
        phi, info = op.advect_levelset(K)
        assert info["converged"] and info["fp_iters"] == K
        ug, flags, _ = op.transport_velocity()
        ug, flags = host(ug).reshape(3, -1), host(flags)
        ugo, flo = transport.transport_velocity(mesh_u, np.clip(prev, -1.0, 1.0), wl.u0, wl.mdot, wl.params)
        assert np.mean(flags == flo) >= 0.98
        ok = (flags == 0) & (flo == 0)
        diff = np.abs(ug[:, ok] - ugo[:, ok]).max(axis=0)
        assert np.mean(diff <= 1e-6 * np.abs(ugo).max()) >= 0.99
        ref = geometry.advection_step(mesh1, wl.phi, ug, wl.params["theta"], wl.params["dt"])
        assert np.linalg.norm(host(phi) - ref) < 1e-10 * np.linalg.norm(wl.phi)
        assert rel(host(phi) - wl.phi, ref - wl.phi) < 1e-7
        prev = host(phi)


def test_advection_tolerance_stops_the_fixed_point():
    """With tol > 0 the passes stop once |phi^(k+1) - phi^(k)| <= tol, well before max_iters; the result is the
    self-consistent level set of the oracle's fixed point (iterated to 1e-9) within the transport parity bar."""
    n = 6
    wl = workloads.random_workload(n, 2, 1, geom="sphere", variant=2, dt=0.05)
    wl.u0 = np.repeat(np.array([0.2, 0.1, -0.1])[:, None], (2 * n + 1) ** 3, axis=1).ravel()
    wl.mdot = np.full((n + 1) ** 3, 200.0)
    op = make_op(wl)
    phi, info = op.advect_levelset(20, tol=1e-9)
    assert info["converged"] and 2 <= info["fp_iters"] < 20 and info["last_change"] <= 1e-9
    ref, _ = geometry.advect_levelset(fe.Mesh(n, 2, 1.0), wl.phi, wl.u0, wl.mdot, wl.params, 8)
    assert rel(host(phi) - wl.phi, ref - wl.phi) < 1e-4
    phi0, info0 = op.advect_levelset(0)
    assert info0["fp_iters"] == 0 and np.array_equal(host(phi0), np.clip(wl.phi, -1, 1))
