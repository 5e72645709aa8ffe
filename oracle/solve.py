"""Definition of the solution of the momentum system (test infrastructure).

The Krylov solve of Table (tab:solver_settings) approximates x = A^{-1} f for the assembled velocity block A of
oracle.momentum (Dirichlet rows are the identity, so x equals f on constrained DoFs).  The oracle states that
definition with a direct sparse factorisation (library routine).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import momentum


def solve(pb: momentum.Problem, f: np.ndarray) -> np.ndarray:
    A = momentum.assemble(pb).tocsc()
    return spla.spsolve(A, f)


def jacobi_diagonal(pb: momentum.Problem) -> np.ndarray:
    return momentum.assemble(pb).diagonal()
