"""Dense direct solves of tiny level systems (TEST INFRASTRUCTURE ONLY).

The level matrix is symmetric positive definite (a weighted graph Laplacian
times dt plus a diagonal >= 1, Sect. 3.1-3.2), so a plain Cholesky
factorisation A = L L^T followed by two triangular solves gives the exact
solution up to rounding, independent of CG.
"""
from __future__ import annotations

import numpy as np


def to_dense(system) -> np.ndarray:
    N = system.N
    A = np.zeros((N, N))
    for i in range(N):
        for k in range(int(system.row_ptr[i]), int(system.row_ptr[i + 1])):
            A[i, int(system.col[k])] += system.val[k]
    return A


def leaf_block(system):
    """(A_ll, b_l, leaf index) restricted to leaf rows/columns."""
    A = to_dense(system)
    idx = np.nonzero(system.leaf)[0]
    return A[np.ix_(idx, idx)], system.b[idx], idx


def cholesky(A: np.ndarray) -> np.ndarray:
    """Textbook column-by-column Cholesky (Golub & Van Loan, Alg. 4.2.1 form)."""
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        s = A[j, j] - np.dot(L[j, :j], L[j, :j])
        if s <= 0.0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        L[j, j] = np.sqrt(s)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def cholesky_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    L = cholesky(A)
    n = len(b)
    y = np.zeros(n)
    for i in range(n):
        y[i] = (b[i] - np.dot(L[i, :i], y[:i])) / L[i, i]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (y[i] - np.dot(L[i + 1:, i], x[i + 1:])) / L[i, i]
    return x
