"""GPU parity of the surface-tension force (Eq. surfaceTension with the density-scaled delta) against the oracle,
through the C ABI.  FP64: relative l2 <= 1e-12 (the same Gauss sums, rounding order only)."""
import numpy as np
import pytest
import torch

import workloads
from oracle import fe, geometry, momentum, surface

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


def make_op(wl):
    from paper_2401_07805_gb300 import Operator
    op = Operator(wl.n, wl.p, wl.L, dict(wl.params))
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    return op


CASES = [("sphere8", dict(name="sphere8")), ("ragged7", dict(n=7, p=2, seed=4, geom="spheres")),
         ("q3_6", dict(n=6, p=3, seed=8, geom="deformed")), ("ratio1e4", dict(n=9, p=2, seed=9, geom="sphere", ratio=1e4))]


@pytest.mark.parametrize("label,kw", CASES, ids=[c[0] for c in CASES])
def test_surface_tension_parity(label, kw):
    if "name" in kw:
        wl = workloads.make_workload(kw["name"])
    else:
        wl = workloads.random_workload(kw["n"], kw["p"], kw["seed"], geom=kw["geom"], ratio=kw.get("ratio", 1e3))
    op = make_op(wl)
    mesh1 = fe.Mesh(wl.n, 1, wl.L)
    nf = geometry.projected_normal(mesh1, wl.phi)
    kappa = geometry.curvature(mesh1, nf)
    f = op.surface_tension(cuda(nf.ravel()), cuda(kappa), 0.0728)
    ref = surface.surface_tension_rhs(momentum.Problem.from_workload(wl), nf, kappa, 0.0728)
    got = f.cpu().numpy()
    assert np.linalg.norm(ref) > 0
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_surface_tension_full_size_from_gpu_geometry():
    """48^3 sphere: normal and curvature from the GPU geometry sub-solver, force from the GPU; the net force of the
    centred drop vanishes (to 1e-10 of the total magnitude) and the force points into the liquid."""
    wl = workloads.make_workload("sphere48")
    op = make_op(wl)
    n, _ = op.projected_normal()
    kappa, _ = op.curvature(n)
    f = op.surface_tension(n, kappa, 1.0).cpu().numpy().reshape(3, -1)
    tot = np.abs(f).sum()
    assert tot > 0 and np.abs(f.sum(axis=1)).max() < 1e-10 * tot
    m = op.n_u
    g = np.arange(round(m ** (1 / 3))) / (round(m ** (1 / 3)) - 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    radial = np.stack([X.ravel() - 0.5, Y.ravel() - 0.5, Z.ravel() - 0.5])
    assert np.sum(f * radial) < 0.0
