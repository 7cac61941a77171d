"""Hand-written dense complex LU with partial pivoting (oracle, test infrastructure).

The paper's linear solver is MATLAB backslash on a dense matrix (Appendix,
linearsolver), i.e. Gaussian elimination with partial pivoting. The pivot in
column k is the row maximising |Re| + |Im| over rows k..n-1, ties going to the
lowest row index (the BLAS izamax convention, which LAPACK zgetrf uses).

Right-looking, unblocked, one column at a time: no blocking or reordering, so
it can be read against the textbook algorithm. Used to cross-check the SciPy
(LAPACK) solves and to pin the GPU pivot sequence on small inputs.
"""
from __future__ import annotations

import numpy as np


def lu_factor_pp(T: np.ndarray):
    """Return (LU, piv) with P T = L U; piv[k] is the row swapped with row k at step k."""
    A = np.array(T, dtype=np.complex128, copy=True)
    n = A.shape[0]
    piv = np.zeros(n, dtype=np.int64)
    for k in range(n):
        col = A[k:, k]
        mag = np.abs(col.real) + np.abs(col.imag)
        p = k + int(np.argmax(mag))          # argmax returns the first (lowest) index on ties
        piv[k] = p
        if p != k:
            A[[k, p], :] = A[[p, k], :]
        if A[k, k] == 0:
            continue                          # exactly singular column: leave it, like LAPACK (info > 0)
        A[k + 1:, k] = A[k + 1:, k] / A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, piv


def lu_solve_pp(LU: np.ndarray, piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve T X = B from lu_factor_pp's output (row swaps, unit-lower then upper substitution)."""
    X = np.array(B, dtype=np.complex128, copy=True)
    n = LU.shape[0]
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    for k in range(n):
        p = piv[k]
        if p != k:
            X[[k, p], :] = X[[p, k], :]
    for i in range(n):                       # L y = P b, L unit lower
        X[i, :] -= LU[i, :i] @ X[:i, :]
    for i in range(n - 1, -1, -1):           # U x = y
        X[i, :] = (X[i, :] - LU[i, i + 1:] @ X[i + 1:, :]) / LU[i, i]
    return X[:, 0] if vec else X
