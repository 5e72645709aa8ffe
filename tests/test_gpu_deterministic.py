"""Deterministic accumulation (evap_set_deterministic): the cells of the operator applies, the adjoint and the Jacobi
diagonal are taken in 8 parity-class passes with plain stores instead of atomic adds.

Checked here: two runs give bitwise identical results (applies at both precisions with the divergence row, the
level-set applies, the adjoint's four gradients, the mixed-precision solve with its iteration count); the results
agree with the oracle at the parity bars of test_gpu_parity (1e-12 FP64, 2e-5 FP32) and with the default atomic mode
to rounding; the colour classes cover every cell once for odd and even cell counts (n = 1, 2, 5, 9) and for the
subdivided level-set mesh.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import adjoint, fe, levelset, momentum, solve

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


def rel(a, b):
    a = a.detach().cpu().numpy() if torch.is_tensor(a) else a
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make_op(wl, deterministic=True):
    from paper_2401_07805_gb300 import Operator
    op = Operator(wl.n, wl.p, wl.L, dict(wl.params))
    op.set_deterministic(deterministic)
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    return op


def same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("n,p", [(1, 2), (2, 2), (5, 2), (9, 2), (5, 3)])
def test_momentum_runs_are_bitwise_identical_and_match_the_oracle(n, p):
    wl = workloads.random_workload(n, p=p, seed=11 + n, geom="sphere")
    op = make_op(wl)
    x = cuda(wl.x)
    y1 = op.apply_momentum(x, prec=64, with_divergence=True)
    y2 = op.apply_momentum(x, prec=64, with_divergence=True)
    assert same(y1, y2)
    pb = momentum.Problem.from_workload(wl)
    yo, ypo = momentum.apply(pb, wl.x, with_divergence=True)
    e, ep = rel(y1[0], yo), rel(y1[1], ypo)
    print(f"deterministic FP64 apply {n}^3 Q{p}: {e:.1e} / {ep:.1e}")
    assert e <= 1e-12 and ep <= 1e-12
    x32 = x.float()
    z1 = op.apply_momentum(x32, prec=32, with_divergence=True)
    z2 = op.apply_momentum(x32, prec=32, with_divergence=True)
    assert same(z1, z2)
    assert rel(z1[0].double(), yo) <= 2e-5 and rel(z1[1].double(), ypo) <= 2e-5
    op.close()


def test_deterministic_and_atomic_modes_agree_to_rounding():
    wl = workloads.random_workload(12, seed=4, geom="spheres")
    a, d = make_op(wl, False), make_op(wl, True)
    x = cuda(wl.x)
    ya, yd = a.apply_momentum(x, prec=64, with_divergence=True), d.apply_momentum(x, prec=64, with_divergence=True)
    assert rel(yd[0], ya[0].cpu().numpy()) <= 1e-14 and rel(yd[1], ya[1].cpu().numpy()) <= 1e-14
    za, zd = a.apply_momentum(x.float(), prec=32), d.apply_momentum(x.float(), prec=32)
    assert rel(zd[0].double(), za[0].double().cpu().numpy()) <= 1e-6
    a.close()
    d.close()


@pytest.mark.parametrize("mode", ["advect", "reinit", "reinit_rhs"])
@pytest.mark.parametrize("prec", [64, 32])
def test_levelset_runs_are_bitwise_identical(mode, prec):
    """Q1 operators on 9^3 with a supplied transport velocity (the oracle's inputs), both precisions."""
    wl = workloads.random_workload(9, seed=5, geom="sphere")
    mesh = fe.Mesh(9, 2, 1.0)
    rng = np.random.default_rng(9)
    ug = rng.uniform(-1.0, 1.0, 3 * mesh.n_phi)
    op = make_op(wl)
    op.set_transport_velocity(cuda(ug))
    x = rng.uniform(-1.0, 1.0, mesh.n_phi) if mode != "reinit_rhs" else wl.phi.copy()
    xin = cuda(x) if prec == 64 else cuda(x).float()
    y1 = op.apply_levelset(xin, mode=mode, prec=prec)
    y2 = op.apply_levelset(xin, mode=mode, prec=prec)
    assert torch.equal(y1, y2)
    xo = x if prec == 64 else x.astype(np.float32).astype(np.float64)
    yo = levelset.apply(mesh, mode, xo, wl.phi, ug, wl.params)
    assert rel(y1.double(), yo) <= (1e-12 if prec == 64 else 2e-5)
    op.close()


@pytest.mark.parametrize("n_sub", [1, 2])
def test_adjoint_runs_are_bitwise_identical_and_match_the_oracle(n_sub):
    wl = workloads.random_workload(6, seed=3, geom="sphere", n_sub=n_sub)
    op = make_op(wl)
    rng = np.random.default_rng(2)
    w = rng.uniform(-1, 1, wl.x.shape)
    wp = rng.uniform(-1, 1, op.n_p)
    g1 = op.apply_adjoint(cuda(w), cuda(wl.x), cuda(wp))
    g2 = op.apply_adjoint(cuda(w), cuda(wl.x), cuda(wp))
    assert all(torch.equal(g1[k], g2[k]) for k in g1)
    pb = momentum.Problem.from_workload(wl)
    gu, gphi, gm = adjoint.param_gradients(pb, wl.x, w, wp)
    errs = dict(x=rel(g1["x"], adjoint.grad_x(pb, w, wp)), u0=rel(g1["u0"], gu), phi=rel(g1["phi"], gphi),
                mdot=rel(g1["mdot"], gm))
    print(f"deterministic adjoint n_sub {n_sub}: " + ", ".join(f"{k} {v:.1e}" for k, v in errs.items()))
    assert max(errs.values()) <= 1e-12
    op.close()


def test_mixed_solve_is_bitwise_reproducible():
    wl = workloads.random_workload(10, seed=6, geom="spheres")
    op = make_op(wl)
    f = cuda(wl.x)
    x1, i1 = op.solve(f, mixed=True, rtol=1e-10)
    x2, i2 = op.solve(f, mixed=True, rtol=1e-10)
    assert torch.equal(x1, x2) and i1["iters"] == i2["iters"]
    pb = momentum.Problem.from_workload(wl)
    assert rel(x1, solve.solve(pb, wl.x)) <= 1e-8
    op.close()
