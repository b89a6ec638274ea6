"""CPU oracle of the LU factorisation and the HPL-style check -- TEST INFRASTRUCTURE ONLY.

Only the tests import this module.  It restates, in plain float64 numpy, what the paper's
HPL run (Section IV-C, Table VII) does with the library's gemm: factor
P A = L U with partial pivoting (L unit lower, U upper; at step j the pivot
is the row of largest |a| in column j on or below the diagonal, the first
such row on ties), solve A x = b, and judge the solution by the scaled
residual HPL prints,
    r = ||A x - b||_inf / (eps (||A||_inf ||x||_inf + ||b||_inf) n),
accepted when r < 16.  Pivots are reported LAPACK style: ipiv[j] (1-based)
is the row swapped with row j at step j.
"""

from __future__ import annotations

import numpy as np


def lu_factor(A: np.ndarray):
    """Right-looking LU with partial pivoting of a square matrix (float64
    copy); returns (LU packed: L below the diagonal, U on and above, ipiv
    1-based, index of the first exactly zero pivot or -1)."""
    a = np.array(A, dtype=np.float64, copy=True)
    n = a.shape[0]
    ipiv = np.zeros(n, dtype=np.int64)
    zero = -1
    for j in range(n):
        p = j + int(np.argmax(np.abs(a[j:, j])))  # first maximum on ties
        ipiv[j] = p + 1
        if p != j:
            a[[j, p], :] = a[[p, j], :]
        if a[j, j] == 0.0:
            if zero < 0:
                zero = j
            continue
        a[j + 1:, j] /= a[j, j]
        a[j + 1:, j + 1:] -= np.outer(a[j + 1:, j], a[j, j + 1:])
    return a, ipiv, zero


def apply_pivots(b: np.ndarray, ipiv: np.ndarray) -> np.ndarray:
    """The row interchanges of ipiv (1-based, in order) applied to b."""
    x = np.array(b, dtype=np.float64, copy=True)
    for j, p in enumerate(ipiv):
        p = int(p) - 1
        if p != j:
            x[[j, p]] = x[[p, j]]
    return x


def lu_solve(lu: np.ndarray, ipiv: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve A x = b from the packed factors: P b, forward substitution with
    unit L, back substitution with U."""
    n = lu.shape[0]
    y = apply_pivots(b, ipiv)
    for i in range(n):
        y[i] -= lu[i, :i] @ y[:i]
    for i in range(n - 1, -1, -1):
        y[i] = (y[i] - lu[i, i + 1:] @ y[i + 1:]) / lu[i, i]
    return y


def unpack(lu: np.ndarray):
    """(L, U) of a packed factorisation."""
    L = np.tril(lu, -1) + np.eye(lu.shape[0])
    U = np.triu(lu)
    return L, U


def permutation(ipiv: np.ndarray, n: int) -> np.ndarray:
    """The row order P (P A = A[order]) produced by the interchanges."""
    return apply_pivots(np.arange(n, dtype=np.float64), ipiv).astype(np.int64)


def hpl_residual(A: np.ndarray, x: np.ndarray, b: np.ndarray, eps: float) -> float:
    """HPL's scaled residual ||A x - b||_inf / (eps (||A||_inf ||x||_inf + ||b||_inf) n), in float64."""
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = A.shape[0]
    r = np.abs(A @ x - b).max()
    den = eps * (np.abs(A).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max()) * n
    return float(r / den)


def factor_residual(A: np.ndarray, lu: np.ndarray, ipiv: np.ndarray, eps: float) -> float:
    """||P A - L U||_inf / (eps ||A||_inf n) of a packed factorisation, in float64."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    L, U = unpack(np.asarray(lu, dtype=np.float64))
    PA = A[permutation(ipiv, n)]
    return float(np.abs(PA - L @ U).sum(axis=1).max() / (eps * np.abs(A).sum(axis=1).max() * n))
