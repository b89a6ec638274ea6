"""Pins of the LU oracle (oracle/lu_ref.py): a 3 x 3 factorisation worked by
hand, agreement with SciPy's LAPACK-backed lu_factor, P A = L U, the solve,
the HPL residual of a case worked by hand, and singular matrices."""

import numpy as np
import pytest

from oracle import lu_ref as L


def test_hand_worked_3x3():
    # A = [[2,1,1],[4,3,3],[8,7,9]].  Step 0: pivot 8 (row 3), l = 1/2, 1/4,
    # rows 2, 3 become [-1/2, -3/2], [-3/4, -5/4].  Step 1: pivot -3/4 (row 3),
    # l = (-1/2)/(-3/4) = 2/3, u22 = -3/2 - (2/3)(-5/4) = -2/3.
    A = np.array([[2, 1, 1], [4, 3, 3], [8, 7, 9]], dtype=np.float64)
    lu, ipiv, zero = L.lu_factor(A)
    want = np.array([[8, 7, 9], [0.25, -0.75, -1.25], [0.5, 2.0 / 3.0, -2.0 / 3.0]])
    assert np.allclose(lu, want, rtol=0, atol=1e-15)
    assert list(ipiv) == [3, 3, 3] and zero == -1


def test_matches_lapack():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(7)
    for n in (1, 5, 40, 129):
        A = rng.uniform(-1, 1, (n, n))
        lu, ipiv, _ = L.lu_factor(A)
        lu2, piv2 = scipy_linalg.lu_factor(A)
        assert np.array_equal(ipiv - 1, piv2)
        assert np.allclose(lu, lu2, rtol=1e-12, atol=1e-12)


def test_reconstruction_and_solve():
    rng = np.random.default_rng(8)
    n = 60
    A = rng.uniform(-1, 1, (n, n))
    lu, ipiv, _ = L.lu_factor(A)
    Lm, Um = L.unpack(lu)
    assert np.allclose(A[L.permutation(ipiv, n)], Lm @ Um, rtol=0, atol=1e-12)
    assert L.factor_residual(A, lu, ipiv, 2.0**-52) < 1.0
    b = rng.uniform(-1, 1, n)
    x = L.lu_solve(lu, ipiv, b)
    assert np.allclose(A @ x, b, rtol=0, atol=1e-10)
    assert L.hpl_residual(A, x, b, 2.0**-52) < 16.0
    # a residual planted in the solution is seen
    assert L.hpl_residual(A, x + 1e-6, b, 2.0**-52) > 16.0


def test_hpl_residual_by_hand():
    eps = 2.0**-24
    # A = [[2]], x = [1], b = [1]: |2 - 1| / (eps (2 * 1 + 1) * 1)
    assert L.hpl_residual(np.array([[2.0]]), np.array([1.0]), np.array([1.0]), eps) == pytest.approx(1.0 / (3 * eps))
    assert L.hpl_residual(np.eye(4), np.arange(4.0), np.arange(4.0), eps) == 0.0


def test_singular_matrix_reports_first_zero_pivot():
    rng = np.random.default_rng(9)
    A = rng.uniform(-1, 1, (8, 8))
    A[:, 5] = 0.0
    _, ipiv, zero = L.lu_factor(A)
    assert zero == 5
