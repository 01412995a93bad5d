"""Dense reference solve of the scaled system (test infrastructure, oracle).

A x = b by LU with partial pivoting (LAPACK zgetrf/zgetrs via SciPy). This is
the exact solution the RS-S factorization approximates (Sec. 4.2, the product
formula for A^{-1}).

Pins: residual ||A x - b|| / ||b|| near machine precision (tests), and the
analytic point-source test of Sec. 6.1 in tests/test_oracle_kernel.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import kernel


def solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    lu = sla.lu_factor(A)
    return sla.lu_solve(lu, b)


def solve_adjoint(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    lu = sla.lu_factor(A)
    return sla.lu_solve(lu, b, trans=2)


def solve_surface(points, normals, weights, k, b, eta=None):
    eta = k if eta is None else eta
    A = kernel.dense_matrix(points, normals, weights, k, eta)
    return solve(A, b), A
