"""Parity at the full workload sizes, in the launch configuration bench.py times.

64^3 four-sphere workload (6.44 M velocity DoFs): the CUDA applies are checked on sampled output rows that the
oracle computes from the cells around the sampled nodes (momentum, divergence row, transport velocity), and the Q1
operators in full.  48^3 sphere workload: the adjoint gradients against central differences (h = 1e-6) of the
loss evaluated by the CUDA forward operator on 50 random directions.  Tolerances as in test_gpu_parity.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import fe, levelset, momentum, physics, transport

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def big():
    import os
    import paper_2401_07805_gb300 as evap
    from paper_2401_07805_gb300 import build
    if not os.path.exists(evap.library_path()):
        build.build()
    wl = workloads.make_workload("spheres64")
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    return wl, op


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _sample_nodes(wl, count, seed):
    """Random Q2 nodes, half of them inside interface cells (phi_h in the zone at the node's Q1 neighbours)."""
    rng = np.random.default_rng(seed)
    m = wl.p * wl.n + 1
    pick = list(rng.integers(0, m ** 3, count // 2))
    q1 = np.nonzero(np.abs(wl.phi) < physics.PHI_BAND)[0]
    m1 = wl.n + 1
    for k in rng.choice(q1, count - len(pick), replace=False):
        i, j, l = k % m1, (k // m1) % m1, k // (m1 * m1)
        pick.append(wl.p * i + m * (wl.p * j + m * wl.p * l))
    pick += [0, m - 1, m * m * m - 1]
    return np.unique(np.array(pick))


def test_momentum_sampled_rows_fp64(big):
    wl, op = big
    y, yp = op.apply_momentum(cuda(wl.x), prec=64, with_divergence=True)
    y = y.cpu().numpy().reshape(3, -1)
    nodes = _sample_nodes(wl, 96, 1)
    pb = momentum.Problem.from_workload(wl)
    yo = momentum.apply_rows(pb, wl.x, nodes)
    assert rel(y[:, nodes], yo) <= 1e-12
    q1n = np.unique(np.concatenate([np.random.default_rng(2).integers(0, op.n_phi, 48),
                                    np.nonzero(np.abs(wl.phi) < physics.PHI_BAND)[0][::997]]))
    ypo = momentum.divergence_rows(pb, wl.x, q1n)
    assert rel(yp.cpu().numpy()[q1n], ypo) <= 1e-12


def test_momentum_sampled_rows_fp32(big):
    wl, op = big
    y = op.apply_momentum(cuda(wl.x).float(), prec=32).double().cpu().numpy().reshape(3, -1)
    nodes = _sample_nodes(wl, 64, 3)
    pb = momentum.Problem.from_workload(wl)
    yo = momentum.apply_rows(pb, wl.x.astype(np.float32).astype(np.float64), nodes)
    assert rel(y[:, nodes], yo) <= 2e-5


def test_levelset_full_64(big):
    import paper_2401_07805_gb300 as evap
    wl, _ = big
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))      # own handle: the transport velocity is overwritten
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    mesh = fe.Mesh(wl.n, wl.p, wl.L)
    rng = np.random.default_rng(9)
    ug = rng.uniform(-1, 1, 3 * op.n_phi)
    op.set_transport_velocity(cuda(ug))
    x = rng.uniform(-1, 1, op.n_phi)
    for mode in ("advect", "reinit", "reinit_rhs"):
        xin = wl.phi if mode == "reinit_rhs" else x
        y = op.apply_levelset(cuda(xin), mode=mode).cpu().numpy()
        assert rel(y, levelset.apply(mesh, mode, xin, wl.phi, ug, wl.params)) <= 1e-12
    op.close()


def test_transport_velocity_sampled_64(big):
    wl, op = big
    ug, flags, nflag = op.transport_velocity()
    ug = ug.cpu().numpy().reshape(3, -1)
    flags = flags.cpu().numpy()
    band = np.nonzero((wl.phi > -physics.PHI_GAS_BAND) & (wl.phi < physics.PHI_BAND))[0]
    rng = np.random.default_rng(4)
    nodes = np.concatenate([rng.choice(band, 160, replace=False), rng.integers(0, op.n_phi, 40)])
    mesh = fe.Mesh(wl.n, wl.p, wl.L)
    ugo, flo = transport.transport_velocity(mesh, wl.phi, wl.u0, wl.mdot, wl.params, nodes=nodes)
    assert np.mean(flags[nodes] == flo) >= 0.98
    ok = (flags[nodes] == 0) & (flo == 0)
    diff = np.abs(ug[:, nodes][:, ok] - ugo[:, ok]).max(axis=0)
    assert np.mean(diff <= 1e-6 * np.abs(ugo).max()) >= 0.99
    assert nflag <= 0.02 * len(band)
    from test_gpu_parity import check_closest_points
    check_closest_points(op, wl, np.asarray(band), sample=1500)


def test_adjoint_finite_differences_48():
    """Gradients of L = w.A(phi, mdot, u0) x + w_p.(B x - g) from the adjoint kernel against central differences
    (h = 1e-6) of L computed by the CUDA forward apply, 50 random directions per argument (seed 1)."""
    import paper_2401_07805_gb300 as evap
    wl = workloads.make_workload("sphere48")
    w, wp = wl.extra["w"], wl.extra["w_p"]
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    fields = dict(phi=wl.phi, u0=wl.u0, mdot=wl.mdot, x=wl.x)

    def loss(absolute=False, **kw):
        f = dict(fields)
        f.update(kw)
        op.set_fields(cuda(f["phi"]), cuda(f["u0"]), cuda(f["mdot"]))
        y, yp = op.apply_momentum(cuda(f["x"]), prec=64, with_divergence=True)
        if absolute:
            return float((cuda(w) * y).abs().sum() + (cuda(wp) * yp).abs().sum())
        return float(cuda(w) @ y + cuda(wp) @ yp)

    l_abs = loss(absolute=True)   # sum of |terms| of L: sets the rounding floor of a difference of two L values
    g = op.apply_adjoint(cuda(w), cuda(wl.x), cuda(wp))
    g = {k: v.cpu().numpy() for k, v in g.items()}
    # phi at the quadrature points, to skip directions whose +-h step crosses the interface-zone edge (the
    # correction term switches on there: L is discontinuous in phi across that edge)
    t = fe.gauss_rule(3)[0]
    mesh = fe.Mesh(wl.n, wl.p, wl.L)
    b1 = fe.tensor_basis(1, t, mesh.h)
    d1 = mesh.dofs_phi()
    rng = np.random.default_rng(1)
    hstep = 1e-6
    # L is linear in mdot, u0 and x: their central differences are exact for any step, so a unit step keeps the
    # rounding of L out of the check; phi enters nonlinearly and takes h = 1e-6.
    for name, key, step in (("phi", "phi", hstep), ("mdot", "mdot", 1.0), ("u0", "u0", 1.0), ("x", "x", 1.0)):
        base = fields[name]
        done = tries = 0
        while done < 50 and tries < 200:
            tries += 1
            v = rng.standard_normal(base.shape)
            if name == "phi":
                lo = np.abs((base - hstep * v)[d1] @ b1.N) < physics.PHI_BAND
                hi = np.abs((base + hstep * v)[d1] @ b1.N) < physics.PHI_BAND
                if np.any(lo != hi):
                    continue
            fd = (loss(**{name: base + step * v}) - loss(**{name: base - step * v})) / (2 * step)
            an = float(g[key] @ v)
            # relative 1e-6, plus the rounding floor of the difference: 1e-14 of sum |terms of L| over 2 step
            assert abs(fd - an) <= 1e-6 * abs(an) + 1e-14 * l_abs / (2 * step), (name, fd, an)
            done += 1
        assert done == 50, (name, done)


@pytest.mark.parametrize("p", [2, 3])
def test_large_case_sampled_rows(p):
    """128^3 cells, degree p (51 M / 171 M velocity DoFs), deformed sphere, density ratio 1e4: sampled rows of the
    FP64 apply (with divergence row) and of the FP32 apply against the oracle."""
    import paper_2401_07805_gb300 as evap
    wl = workloads.make_workload("deformed128", p=p)
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    x = cuda(wl.x)
    y, yp = op.apply_momentum(x, prec=64, with_divergence=True)
    nodes = _sample_nodes(wl, 48, 11)
    pb = momentum.Problem.from_workload(wl)
    yo = momentum.apply_rows(pb, wl.x, nodes)
    y = y.view(3, -1)
    assert rel(y[:, nodes].cpu().numpy(), yo) <= 1e-12
    q1n = np.unique(np.concatenate([np.random.default_rng(5).integers(0, op.n_phi, 24),
                                    np.nonzero(np.abs(wl.phi) < physics.PHI_BAND)[0][::4999]]))
    assert rel(yp.cpu().numpy()[q1n], momentum.divergence_rows(pb, wl.x, q1n)) <= 1e-12
    del y, yp
    y32 = op.apply_momentum(x.float(), prec=32).view(3, -1)
    yo32 = momentum.apply_rows(pb, wl.x.astype(np.float32).astype(np.float64), nodes)
    assert rel(y32[:, nodes].double().cpu().numpy(), yo32) <= 2e-5
    op.close()
    torch.cuda.empty_cache()
