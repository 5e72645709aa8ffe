"""GPU parity: every CUDA operator against the CPU oracle on the same seeded inputs, element by element.

Tolerances (relative l2 unless stated), written per test:
  * FP64 applies and adjoint: <= 1e-12 (the target of the method; both sides evaluate the same Gauss sums and
    differ only in rounding order);
  * FP32 applies: <= 2e-5 (unit roundoff 6e-8 times the depth of the sums: 3 sweeps in, ~12-term fluxes, 3 sweeps
    out, over a ~1e7 spread between the mass and viscous coefficients);
  * transport velocity: variant 1 (no iteration) to 1e-13 of the velocity scale; variants 2/3: the closest-point
    iteration stops when no shorter point is found, a decision taken at rounding level near the minimum, and on
    creases of the discrete isocontour it can reach another local minimum; the oracle itself moves ~4 % of the
    nodes by more than 1e-9 and ~0.2 % by more than 1e-3 under 1-ulp input perturbations
    (test_oracle_pins.test_closest_point_rounding_sensitivity).  Bar: flags agree on >= 98 % of nodes and >= 99 %
    of the nodes unflagged on both sides agree to 1e-6 of the velocity scale;
  * solves: the solution error against the oracle's direct solve, <= 1e-9 (FP64, rtol 1e-12) and <= 1e-8
    (mixed precision, rtol 1e-10).
Sizes span several thread blocks with a ragged last block (cells per block: 8 for Q2, 4 for Q3).
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import adjoint, fe, levelset, momentum, solve, transport

pytestmark = pytest.mark.gpu


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


def make_op(wl):
    from paper_2401_07805_gb300 import Operator
    op = Operator(wl.n, wl.p, wl.L, dict(wl.params))
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    return op


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------------------------------------------- momentum
def test_momentum_fp64_sphere8():
    """Plain FP64 apply on 8^3 cells (sphere, ratio 1e3, u and x from seed 0) against the assembled oracle."""
    wl = workloads.make_workload("sphere8")
    op = make_op(wl)
    y, yp = op.apply_momentum(cuda(wl.x), prec=64, with_divergence=True)
    pb = momentum.Problem.from_workload(wl)
    yo, ypo = momentum.apply(pb, wl.x, with_divergence=True)
    assert rel(y, yo) <= 1e-12
    assert rel(yp, ypo) <= 1e-12


CASES = [  # n, p, geom, overrides
    (1, 2, "sphere", dict(dirichlet_faces=0)),
    (3, 2, "sphere", dict()),
    (5, 2, "slab", dict(newton=0, stress=0)),
    # correction everywhere needs a level-set gradient that vanishes nowhere (n = grad phi/|grad phi| is undefined
    # where it is at rounding level, e.g. the centre cell of a symmetric sphere): slab with a wide profile
    (5, 2, "slab", dict(corr_zone=1, dirichlet_faces=0x15, eps=0.3)),
    (7, 2, "spheres", dict(ratio=1e4)),
    (2, 3, "sphere", dict(dirichlet_faces=0)),
    (3, 3, "sphere", dict(corr_zone=1)),
    (5, 3, "slab", dict(dirichlet_faces=0x2A)),
]


def _case(n, p, geom, over, seed=0):
    over = dict(over)
    ratio = over.pop("ratio", 1e3)
    wl = workloads.random_workload(n, p=p, seed=seed + n, geom=geom, ratio=ratio, **over)
    if n <= 3:
        wl.params["eps"] = 0.3          # coarse meshes: keep most points inside the interface zone
        rng = np.random.default_rng(seed)
        wl.phi = rng.uniform(-0.95, 0.95, wl.phi.shape)
    return wl


@pytest.mark.parametrize("n,p,geom,over", CASES)
def test_momentum_fp64_cases(n, p, geom, over):
    wl = _case(n, p, geom, over)
    op = make_op(wl)
    y, yp = op.apply_momentum(cuda(wl.x), prec=64, with_divergence=True)
    pb = momentum.Problem.from_workload(wl)
    yo, ypo = momentum.apply(pb, wl.x, with_divergence=True)
    assert rel(y, yo) <= 1e-12
    assert rel(yp, ypo) <= 1e-12


@pytest.mark.parametrize("n,p,geom,over", CASES[1:6])
def test_momentum_fp32_cases(n, p, geom, over):
    wl = _case(n, p, geom, over)
    op = make_op(wl)
    y, yp = op.apply_momentum(cuda(wl.x).float(), prec=32, with_divergence=True)
    assert y.dtype == torch.float32
    pb = momentum.Problem.from_workload(wl)
    yo, ypo = momentum.apply(pb, wl.x.astype(np.float32).astype(np.float64), with_divergence=True)
    assert rel(y.double(), yo) <= 2e-5
    assert rel(yp.double(), ypo) <= 2e-5


def test_momentum_pure_phases_and_zero_mass_flux():
    """No interface cell at all (phi = 1) and mdot = 0: constants path of the kernel, divergence row without source."""
    wl = workloads.random_workload(4, seed=3)
    wl.phi = np.ones_like(wl.phi)
    wl.mdot = np.zeros_like(wl.mdot)
    op = make_op(wl)
    y, yp = op.apply_momentum(cuda(wl.x), prec=64, with_divergence=True)
    pb = momentum.Problem.from_workload(wl)
    yo, ypo = momentum.apply(pb, wl.x, with_divergence=True)
    assert rel(y, yo) <= 1e-12 and rel(yp, ypo) <= 1e-12


def test_single_cell_all_dirichlet():
    """One Q2 cell with all faces constrained: 26 boundary nodes pass x through, the centre node is a real row."""
    wl = workloads.random_workload(1, seed=1)
    op = make_op(wl)
    y = op.apply_momentum(cuda(wl.x), prec=64).cpu().numpy()
    pb = momentum.Problem.from_workload(wl)
    mask = pb.constrained()
    np.testing.assert_array_equal(y[mask], wl.x[mask])
    yo = momentum.apply(pb, wl.x)
    assert rel(y[~mask], yo[~mask]) <= 1e-12


# --------------------------------------------------------------------------------------------------- level set
@pytest.mark.parametrize("mode", ["advect", "reinit", "reinit_rhs"])
@pytest.mark.parametrize("prec", [64, 32])
def test_levelset_sphere8(mode, prec):
    """Q1 operators on 8^3 with the transport velocity supplied to both sides (the oracle's u_Gamma at 8^3)."""
    wl = workloads.make_workload("sphere8")
    mesh = fe.Mesh(8, 2, 1.0)
    rng = np.random.default_rng(4)
    ug = rng.uniform(-1.0, 1.0, 3 * mesh.n_phi)
    op = make_op(wl)
    op.set_transport_velocity(cuda(ug))
    x = rng.uniform(-1.0, 1.0, mesh.n_phi) if mode != "reinit_rhs" else wl.phi.copy()
    xin = cuda(x) if prec == 64 else cuda(x).float()
    y = op.apply_levelset(xin, mode=mode, prec=prec)
    xo = x if prec == 64 else x.astype(np.float32).astype(np.float64)
    yo = levelset.apply(mesh, mode, xo, wl.phi, ug, wl.params)
    assert rel(y.double(), yo) <= (1e-12 if prec == 64 else 2e-5)


@pytest.mark.parametrize("n", [1, 5, 11])
def test_levelset_ragged(n):
    wl = workloads.random_workload(n, seed=7, geom="slab")
    mesh = fe.Mesh(n, 2, 1.0)
    rng = np.random.default_rng(n)
    ug = rng.uniform(-1.0, 1.0, 3 * mesh.n_phi)
    op = make_op(wl)
    op.set_transport_velocity(cuda(ug))
    x = rng.uniform(-1.0, 1.0, mesh.n_phi)
    for mode in ("advect", "reinit", "reinit_rhs"):
        y = op.apply_levelset(cuda(x), mode=mode)
        assert rel(y, levelset.apply(mesh, mode, x, wl.phi, ug, wl.params)) <= 1e-12


# ------------------------------------------------------------------------------------------ transport velocity
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_transport_velocity(variant):
    n = 16
    wl = workloads.random_workload(n, seed=5, geom="sphere", variant=variant)
    q1 = workloads.node_coords(n, 1)
    wl.phi = np.tanh(workloads.signed_distance("sphere", q1, radius=0.3) / (2 * wl.params["eps"]))
    op = make_op(wl)
    ug, flags, nflag = op.transport_velocity()
    ug = ug.cpu().numpy().reshape(3, -1)
    flags = flags.cpu().numpy()
    assert nflag == int(flags.sum())
    mesh = fe.Mesh(n, 2, 1.0)
    ugo, flo = transport.transport_velocity(mesh, wl.phi, wl.u0, wl.mdot, wl.params)
    assert np.mean(flags == flo) >= 0.98
    ok = (flags == 0) & (flo == 0)
    scale = np.abs(ugo).max()
    diff = np.abs(ug[:, ok] - ugo[:, ok]).max(axis=0)
    if variant == 1:   # no iteration: plain formula at the node
        assert nflag == 0 and diff.max() <= 1e-13 * scale
    else:              # iteration stops at its own resolution; crease nodes may end at another local minimum
        assert np.mean(diff <= 1e-6 * scale) >= 0.99
        check_closest_points(op, wl, np.nonzero(flags >= 0)[0], every_oracle=True)


def check_closest_points(op, wl, nodes, every_oracle=True, sample=None):
    """Every GPU closest point on its own terms (App. C), for the projection-band nodes among ``nodes``:
      (a) u_Gamma is the variant's formula evaluated at the GPU's point y (u(y) + mdot / rho_* n(x)), to rounding,
          for flagged nodes too;
      (b) an unflagged y lies on the isocontour d(phi_h(y)) = d* (+-3 eps) to the projection's tolerance;
      (c) an unflagged y is no farther from the node than the oracle's unflagged closest point (+ 1e-6 h): where the
          two differ (creases of the piecewise-trilinear isocontour, ties), the GPU's point is at least as close;
      (d) y - x is normal to the isocontour at y (its tangential part at most 1e-3 |y - x|) except at crease
          points; the share of such nodes is at most the oracle's own share plus 1 %.
    (c) and (d) compare with the oracle's points on all band nodes, or on a random sample of ``sample`` of them."""
    from oracle import physics
    prm = wl.params
    mesh = fe.Mesh(wl.n, wl.p, wl.L, int(prm.get("n_sub", 1)))
    variant = int(prm["variant"])
    eps, h = prm["eps"], mesh.h / mesh.n_sub  # cell units of the level-set mesh
    d_t = 3.0 * eps if variant == 2 else -3.0 * eps
    rho_t = prm["rho_l"] if variant == 2 else prm["rho_g"]
    ug, flags, _ = op.transport_velocity()
    ug = ug.cpu().numpy().reshape(3, -1)
    flags = flags.cpu().numpy()
    y = op.closest_points().cpu().numpy() / h                      # cell units
    m1 = mesh.n * mesh.n_sub + 1
    phi = wl.phi
    if variant == 2:
        band = (-physics.PHI_GAS_BAND < phi) & (phi < physics.PHI_BAND)
    else:
        band = (-physics.PHI_BAND < phi) & (phi < physics.PHI_GAS_BAND)
    nodes = np.asarray([k for k in nodes if band[k]])
    assert len(nodes) > 0
    ev = transport.PointEval(mesh, phi, wl.u0)
    scale = max(np.abs(ug).max(), 1e-300)
    xs = np.stack([nodes % m1, (nodes // m1) % m1, nodes // (m1 * m1)]).astype(float)
    for t, node in enumerate(nodes):
        s = y[:, node]
        _, gx = ev.phi_grad(xs[:, t])
        expect = ev.velocity(s) + wl.mdot[node] / rho_t * physics.normal(gx, h)
        assert np.abs(ug[:, node] - expect).max() <= 1e-12 * scale, node                       # (a)
        if flags[node] == 0:
            ph = min(max(ev.phi_grad(s)[0], -transport.PHI_CLAMP), transport.PHI_CLAMP)
            assert abs(float(physics.distance(ph, eps)) - d_t) <= 1e-8 * h, node               # (b)
    rng = np.random.default_rng(0)
    cmp = nodes if sample is None or sample >= len(nodes) else rng.choice(nodes, sample, replace=False)
    _, flo, yo = transport.transport_velocity(mesh, phi, wl.u0, wl.mdot, prm, nodes=cmp, return_points=True)
    xc = np.stack([cmp % m1, (cmp // m1) % m1, cmp // (m1 * m1)]).astype(float)
    both = (flags[cmp] == 0) & (flo == 0)
    dg = np.linalg.norm(y[:, cmp] - xc, axis=0)
    do = np.linalg.norm(yo - xc, axis=0)
    assert np.all(dg[both] <= do[both] + 1e-6), np.max(dg[both] - do[both])                      # (c)

    def tangential_share(pts, sel):
        bad = 0
        for t in np.nonzero(sel)[0]:
            tp = transport.tangential_part(ev, xc[:, t], pts[:, t])
            dist = np.linalg.norm(pts[:, t] - xc[:, t])
            bad += np.linalg.norm(tp) > 1e-3 * dist + 1e-9
        return bad / max(int(sel.sum()), 1)

    share_g = tangential_share(y[:, cmp], flags[cmp] == 0)
    share_o = tangential_share(yo, flo == 0)
    print(f"closest points: {len(nodes)} band nodes checked, {len(cmp)} against the oracle; off-normal share "
          f"GPU {share_g:.4f}, oracle {share_o:.4f}")
    assert share_g <= share_o + 0.01                                                            # (d)


# ---------------------------------------------------------------------------------------------------- adjoint
@pytest.mark.parametrize("case", ["sphere8", "q3", "everywhere", "picard"])
def test_adjoint_against_oracle(case):
    """g_x against the oracle's explicit transposes A^T w + B^T w_p; g_u0, g_phi, g_mdot against its chain rule."""
    if case == "sphere8":
        wl = workloads.make_workload("sphere8")
    elif case == "q3":
        wl = _case(3, 3, "sphere", dict())
    elif case == "everywhere":
        wl = _case(3, 2, "sphere", dict(corr_zone=1))
    else:
        wl = _case(4, 2, "slab", dict(newton=0, stress=0))
    rng = np.random.default_rng(12)
    w = rng.uniform(-1, 1, wl.x.shape)
    wp = rng.uniform(-1, 1, wl.phi.shape)
    op = make_op(wl)
    g = op.apply_adjoint(cuda(w), cuda(wl.x), cuda(wp))
    pb = momentum.Problem.from_workload(wl)
    gx = adjoint.grad_x(pb, w, wp)
    gu, gphi, gm = adjoint.param_gradients(pb, wl.x, w, wp)
    errs = dict(x=rel(g["x"], gx), u0=rel(g["u0"], gu), phi=rel(g["phi"], gphi), mdot=rel(g["mdot"], gm))
    g2 = op.apply_adjoint(cuda(w), cuda(wl.x), None, need=("x", "phi"))  # without the divergence row
    errs.update(x_nodiv=rel(g2["x"], adjoint.grad_x(pb, w)),
                phi_nodiv=rel(g2["phi"], adjoint.param_gradients(pb, wl.x, w)[1]))
    print("adjoint", case, " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v <= 1e-12, (k, v)
    assert g2["u0"] is None and g2["mdot"] is None


def test_autograd_function_matches_adjoint():
    from paper_2401_07805_gb300 import MomentumFunction
    wl = workloads.make_workload("sphere8")
    op = make_op(wl)
    x = cuda(wl.x).requires_grad_(True)
    phi = cuda(wl.phi).requires_grad_(True)
    u0 = cuda(wl.u0).requires_grad_(True)
    md = cuda(wl.mdot).requires_grad_(True)
    y, yp = MomentumFunction.apply(op, x, phi, u0, md)
    rng = np.random.default_rng(2)
    w, wp = cuda(rng.uniform(-1, 1, wl.x.shape)), cuda(rng.uniform(-1, 1, wl.phi.shape))
    ((y * w).sum() + (yp * wp).sum()).backward()
    pb = momentum.Problem.from_workload(wl)
    assert rel(x.grad, adjoint.grad_x(pb, w.cpu().numpy(), wp.cpu().numpy())) <= 1e-12
    gu, gphi, gm = adjoint.param_gradients(pb, wl.x, w.cpu().numpy(), wp.cpu().numpy())
    assert rel(phi.grad, gphi) <= 1e-12 and rel(u0.grad, gu) <= 1e-12 and rel(md.grad, gm) <= 1e-12


def test_autograd_two_forwards_then_backward():
    """Two forwards on the same operator with different fields, then backward through the first: its gradients are
    taken at the first forward's fields (the second set_fields must not leak into them)."""
    from paper_2401_07805_gb300 import MomentumFunction
    wl = workloads.make_workload("sphere8")
    wl2 = workloads.random_workload(8, seed=3, geom="spheres")
    op = make_op(wl)
    x = cuda(wl.x).requires_grad_(True)
    phi = cuda(wl.phi).requires_grad_(True)
    u0 = cuda(wl.u0).requires_grad_(True)
    md = cuda(wl.mdot).requires_grad_(True)
    y, yp = MomentumFunction.apply(op, x, phi, u0, md)
    y2, _ = MomentumFunction.apply(op, cuda(wl2.x), cuda(wl2.phi), cuda(wl2.u0), cuda(wl2.mdot))
    rng = np.random.default_rng(2)
    w, wp = cuda(rng.uniform(-1, 1, wl.x.shape)), cuda(rng.uniform(-1, 1, wl.phi.shape))
    ((y * w).sum() + (yp * wp).sum()).backward()
    pb = momentum.Problem.from_workload(wl)
    assert rel(x.grad, adjoint.grad_x(pb, w.cpu().numpy(), wp.cpu().numpy())) <= 1e-12
    gu, gphi, gm = adjoint.param_gradients(pb, wl.x, w.cpu().numpy(), wp.cpu().numpy())
    assert rel(phi.grad, gphi) <= 1e-12 and rel(u0.grad, gu) <= 1e-12 and rel(md.grad, gm) <= 1e-12


# ------------------------------------------------------------------------------------------------------ solve
def test_jacobi_diagonal():
    wl = workloads.make_workload("sphere8")
    op = make_op(wl)
    d = op.jacobi_diagonal().cpu().numpy()
    do = solve.jacobi_diagonal(momentum.Problem.from_workload(wl))
    np.testing.assert_allclose(d, do, rtol=2e-5)


SOLVE_CASES = [(6, 2, None), (4, 3, 0x2A), (5, 2, 0), (5, 2, 0x1F)]


@pytest.mark.parametrize("n,p,faces", SOLVE_CASES, ids=["q2_box", "q3_mixed_faces", "q2_no_faces", "q2_open_top"])
@pytest.mark.parametrize("mixed", [False, True])
def test_solve_against_direct(mixed, n, p, faces):
    """Both solves (FP64 GMRES and the mixed one) with the tensor-product mass preconditioner, whose line solves
    run over the free node range of each axis (set by the Dirichlet faces) and whose factors have bandwidth p."""
    over = {} if faces is None else dict(dirichlet_faces=faces)
    wl = workloads.make_workload("sphere8", n=n, p=p, **over)
    op = make_op(wl)
    rng = np.random.default_rng(3)
    f = rng.uniform(-1, 1, wl.x.shape)
    x, info = op.solve(cuda(f), mixed=mixed, restart=30, rtol=1e-12 if not mixed else 1e-10, max_iter=3000)
    assert info["converged"], info
    xo = solve.solve(momentum.Problem.from_workload(wl), f)
    assert rel(x, xo) <= (1e-9 if not mixed else 1e-8)
    # the reported residual is the true FP64 residual
    r = op.apply_momentum(x, prec=64) - cuda(f)
    assert abs(r.norm().item() / np.linalg.norm(f) - info["relres"]) <= 1e-3 * info["relres"] + 1e-15


def test_solve_zero_rhs_and_cap():
    wl = workloads.make_workload("sphere8", n=4)
    op = make_op(wl)
    x, info = op.solve(torch.zeros(3 * op.n_u, dtype=torch.float64, device="cuda"), mixed=True)
    assert info["converged"] and info["iters"] == 0 and float(x.abs().max()) == 0.0
    f = cuda(np.random.default_rng(0).uniform(-1, 1, 3 * op.n_u))
    x, info = op.solve(f, mixed=False, rtol=1e-14, max_iter=2)
    assert not info["converged"] and info["iters"] <= 3


# -------------------------------------------------------------------------------------------- error handling
def test_status_codes():
    from paper_2401_07805_gb300 import EvapError, Operator
    op = Operator(4, 2, 1.0, {})
    x = torch.zeros(3 * op.n_u, dtype=torch.float64, device="cuda")
    with pytest.raises(EvapError) as e:
        op.apply_momentum(x)
    assert e.value.status == -4           # fields not set
    wl = workloads.random_workload(4)
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    from paper_2401_07805_gb300 import lib
    import ctypes
    assert lib().evap_apply_momentum(op._h, 16, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr() + 8),
                                     None, None) == -1
    assert lib().evap_apply_levelset(op._h, 9, 64, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr() + 8),
                                     None) == -1
