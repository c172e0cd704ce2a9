"""Naive dense LU with partial pivoting and the triangular solves (Section 6:
each mode is factored by Gaussian elimination).

Pivot = entry of largest complex modulus in the column; ties go to the
lowest row index (numpy's argmax returns the first maximum)."""
from __future__ import annotations

import numpy as np


def lu_factor(A, steps=None):
    """In-place-style LU of a copy of A: returns (LU, piv) with P A = L U,
    L unit lower triangular stored below the diagonal.  ``steps`` stops the
    elimination after that many columns (used to time a sample of it)."""
    A = np.array(A, dtype=complex, copy=True)
    n = A.shape[0]
    piv = np.arange(n)
    for k in range(n if steps is None else min(int(steps), n)):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if A[p, k] == 0:
            raise ZeroDivisionError(f"exact zero pivot in column {k}")
        if p != k:
            A[[k, p], :] = A[[p, k], :]
            piv[[k, p]] = piv[[p, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, piv


def lu_solve(LU, piv, b):
    """Solve A x = b given P A = L U (b may be [n] or [n, nrhs])."""
    x = np.array(b, dtype=complex, copy=True)[piv]
    n = LU.shape[0]
    for k in range(n):                       # forward, unit diagonal
        x[k + 1:] -= np.multiply.outer(LU[k + 1:, k], x[k])
    for k in range(n - 1, -1, -1):           # backward
        x[k] /= LU[k, k]
        x[:k] -= np.multiply.outer(LU[:k, k], x[k])
    return x
