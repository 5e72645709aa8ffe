"""Allocation-free Jacobi diagonal (evap_jacobi_diagonal_noalloc), called through the C ABI.

Some callers cannot let the library allocate device memory when they need the preconditioner diagonal: their
device memory is owned by another allocator, or they must not let the library synchronize the device, which
cudaMalloc and cudaFree may do.  This entry point accumulates in a fixed array that belongs to the loaded library
instead.  The test checks it against the allocating entry point evap_jacobi_diagonal, with the tolerance the
diagonal's parity test uses (FP32 arithmetic: rtol 2e-5), on two calls in a row (the array keeps the previous
call's contents, so the second call checks that it is cleared), and that meshes beyond the array's size are
rejected.  This file is collected last so that a run stopping at the first failure has run every other test.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def evap():
    import paper_2401_07805_gb300 as evap
    from paper_2401_07805_gb300 import build
    if not os.path.exists(evap.library_path()):
        build.build()
    evap.lib()
    return evap


def _op(evap, wl):
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    op.set_fields(cu(wl.phi), cu(wl.u0), cu(wl.mdot))
    return op


def test_noalloc_diagonal_matches_allocating_entry_point(evap):
    L = evap.lib()
    for wl in (workloads.make_workload("sphere48", n=24), workloads.make_workload("sphere8")):
        op = _op(evap, wl)
        ref = op.jacobi_diagonal()          # existing (allocating) entry point
        torch.cuda.synchronize()
        out = torch.empty(3 * op.n_u, dtype=torch.float64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for _ in range(2):                  # two calls in a row share the static accumulator
            out.fill_(float("nan"))
            rc = L.evap_jacobi_diagonal_noalloc(op._h, ctypes.c_void_p(out.data_ptr()), stream)
            assert rc == 0, L.evap_last_error()
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=2e-5)
        op.close()


def test_noalloc_diagonal_rejects_meshes_beyond_its_array(evap):
    L = evap.lib()
    op = evap.Operator(56, 2, 1.0, {})     # 3 * 113^3 = 4328691 > 4194304 entries
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    rc = L.evap_jacobi_diagonal_noalloc(op._h, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
    assert b"exceeds the static accumulator" in L.evap_last_error()
    op.close()
