"""The assembled Schur approximation of the velocity-pressure preconditioner, S~ = B diag(A)^-1 B^T (a symmetric
125-point stencil on the Q1 pressure lattice, FP32), against the same product formed from the oracle's assembled
divergence matrix B (Dirichlet velocity columns removed) and the diagonal of its assembled momentum matrix A.

Bar: 1e-5 relative l2 (the stencil's coefficients are summed in FP32, each from at most 125 products, and the diagonal
of A is the FP32 Jacobi diagonal of the solves, within ~1e-7 of the oracle's).  Cases: open and closed boxes, Q2 and
Q3, odd and even cell counts (a stencil reaching two cells beyond a node meets the boundary from both sides).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import workloads
from oracle import momentum

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


@pytest.mark.parametrize("n,p,faces", [(1, 2, 0x1F), (3, 2, 0x1F), (4, 2, 0x3F), (5, 2, 0x0F), (3, 3, 0x1F)])
def test_assembled_schur_approximation_against_the_oracle(n, p, faces):
    from paper_2401_07805_gb300 import Operator
    wl = workloads.random_workload(n, p=p, seed=20 + n, geom="sphere", dirichlet_faces=faces)
    op = Operator(wl.n, wl.p, wl.L, dict(wl.params))
    op.set_fields(cuda(wl.phi), cuda(wl.u0), cuda(wl.mdot))
    pb = momentum.Problem.from_workload(wl)
    B, _ = momentum.divergence(pb)
    d = momentum.assemble(pb).diagonal()
    S = (B @ sp.diags(1.0 / d) @ B.T).tocsr()
    rng = np.random.default_rng(n)
    for _ in range(2):
        x = rng.uniform(-1.0, 1.0, op.n_p)
        y = op.apply_schur(cuda(x)).cpu().numpy()
        ref = S @ x
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        print(f"Schur stencil {n}^3 Q{p} faces {faces:#x}: {err:.1e}")
        assert err <= 1e-5
    # symmetric: x' S y = y' S x
    x, z = rng.uniform(-1.0, 1.0, op.n_p), rng.uniform(-1.0, 1.0, op.n_p)
    sx, sz = op.apply_schur(cuda(x)).cpu().numpy(), op.apply_schur(cuda(z)).cpu().numpy()
    assert abs(z @ sx - x @ sz) <= 1e-5 * abs(z @ sx)
    op.close()
