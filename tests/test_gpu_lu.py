"""GPU parity of the LU factorisation and solve (gbgemm_sgetrf / gbgemm_sgetrs)
against the FP64 oracle of oracle/lu_ref.py: the HPL run of the paper
(Section IV-C, Table VII).

Where the result is unique the comparison is exact or elementwise: matrices
built as A = P^T L U with |l_ij| small fix every pivot by a wide margin, so
ipiv must equal the oracle's bit for bit and the factors must agree within
a bound on FP32 rounding.  On random matrices pivots can legitimately differ
from FP64 in near-ties, so there the checks are the properties any correct
answer has: the normwise backward error ||P A - L U|| / (eps ||A|| n) and
HPL's scaled residual, both below HPL's threshold 16 with eps = 2^-24.
"""

import numpy as np
import pytest

from oracle import lu_ref as O
from paper_1608_05265_gb300 import synth

from gpu_util import dev

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def h():
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    hd = gbgemm.Handle(0)
    hd.set_stream(torch.cuda.current_stream())
    yield hd
    hd.close()


def factor(h, A_flat, n, lda, nb=0):
    """Run sgetrf on a copy of A (column-major flat, leading dimension lda);
    returns (packed factors as n x n float64, ipiv, info, raw output)."""
    import torch
    dA = dev(A_flat)
    ipiv = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    h.sgetrf(n, dA, lda, ipiv, info, nb)
    torch.cuda.synchronize()
    assert h.get_device_status() == 0
    out = dA.cpu().numpy()
    lu = synth.logical(out, n, n, lda).astype(np.float64) if n > 0 else np.zeros((0, 0))
    return lu, ipiv.cpu().numpy()[:n].astype(np.int64), int(info.item()), out


def solve(h, lu_flat, n, lda, ipiv, B):
    import torch
    dLU = dev(lu_flat)
    dP = torch.from_numpy(ipiv.astype(np.int32)).cuda()
    dB = dev(B)
    nrhs = B.shape[0] if B.ndim == 2 else 1
    h.sgetrs(n, nrhs, dLU, lda, dP, dB, n)
    torch.cuda.synchronize()
    return dB.cpu().numpy().astype(np.float64)


def clear_pivot_matrix(seed, n):
    """A = P^T L U with |l_ij| <= 0.5 / sqrt(n), diag(U) in [1, 2] and
    |u_ij| <= 1 / sqrt(n): partial pivoting must pick, at every step, the row
    P puts there (its candidate is |u_jj|, every other at most half of it)."""
    s = 1.0 / np.sqrt(max(n, 1))
    Lw = 0.5 * s * synth.uniform_pm1(synth.draws(seed, 10, n * n)).reshape(n, n).astype(np.float64)
    Uw = s * synth.uniform_pm1(synth.draws(seed, 11, n * n)).reshape(n, n).astype(np.float64)
    d = 1.5 + 0.5 * synth.uniform_pm1(synth.draws(seed, 12, max(n, 1)))[:n].astype(np.float64)
    L = np.tril(Lw, -1) + np.eye(n)
    U = np.triu(Uw, 1) + np.diag(d)
    order = np.argsort(synth.draws(seed, 13, max(n, 1))[:n], kind="stable")
    A = np.empty((n, n))
    A[order] = L @ U  # row order[i] of A is row i of L U
    return A.astype(np.float32)


def colmajor(A, lda):
    n = A.shape[0]
    return synth.place_colmajor(np.ascontiguousarray(A.T).reshape(-1), n, A.shape[1], lda)


@pytest.mark.parametrize("n,nb", [(1, 0), (2, 1), (9, 0), (9, 8), (40, 7), (40, 0), (130, 32), (130, 128),
                                  (300, 0), (300, 13), (300, 64), (300, 128), (517, 96)])
def test_clear_pivots_match_oracle(h, n, nb):
    A = clear_pivot_matrix(100 + n, n)
    lda = n + 3
    lu, ipiv, info, out = factor(h, colmajor(A, lda), n, lda, nb)
    assert synth.padding_is_sentinel(out, n, n, lda), "write outside the logical matrix"
    want, wpiv, zero = O.lu_factor(A.astype(np.float64))
    assert zero == -1 and info == 0
    assert np.array_equal(ipiv, wpiv), "pivot sequence differs from the oracle"
    # |L|, |U| = O(1) and well conditioned: the FP32 factors agree with the
    # FP64 ones to a few n eps; 16 n eps leaves a wide margin
    assert np.max(np.abs(lu - want)) <= 16 * n * EPS32


@pytest.mark.parametrize("n,nb", [(1, 0), (3, 0), (64, 0), (100, 8), (257, 0), (257, 33), (600, 0), (600, 128),
                                  (1000, 64)])
def test_random_residuals(h, n, nb):
    lda = n + 5
    Af = synth.uniform_matrix(7 + n, 0, n, n, lda)
    A = synth.logical(Af, n, n, lda).astype(np.float64)
    lu, ipiv, info, out = factor(h, Af, n, lda, nb)
    assert info == 0
    assert synth.padding_is_sentinel(out, n, n, lda)
    assert all(j + 1 <= p <= n for j, p in enumerate(ipiv)), "ipiv out of range"
    Lm, Um = O.unpack(lu)
    # partial pivoting keeps |l_ij| <= 1; scaling by the reciprocal adds one rounding
    assert np.max(np.abs(np.tril(lu, -1))) <= 1.0 + 2.0 ** -23
    assert O.factor_residual(A, lu, ipiv, EPS32) < 16
    b = synth.uniform_pm1(synth.draws(7 + n, 5, n)).astype(np.float32)
    x = solve(h, out, n, lda, ipiv, b)
    assert O.hpl_residual(A, x, b.astype(np.float64), EPS32) < 16


def test_hpl_size_of_the_paper(h):
    """N = 4608 (the paper's HPL run), default panel width, three right-hand sides."""
    n = 4608
    Af = synth.uniform_matrix(4608, 0, n, n, n)
    A = synth.logical(Af, n, n, n).astype(np.float64)
    lu, ipiv, info, out = factor(h, Af, n, n)
    assert info == 0
    assert O.factor_residual(A, lu, ipiv, EPS32) < 16
    B = np.stack([synth.uniform_pm1(synth.draws(4608, 5 + r, n)) for r in range(3)]).astype(np.float32)
    X = solve(h, out, n, n, ipiv, B)
    for r in range(3):
        assert O.hpl_residual(A, X[r], B[r].astype(np.float64), EPS32) < 16


def test_cluster_sizes(h):
    """n = 6400: panels on clusters of 16 blocks while a block of 8 would
    hold more than 512 rows, then of 8, and on a single block for the last
    256 rows."""
    n = 6400
    Af = synth.uniform_matrix(6400, 0, n, n, n)
    A = synth.logical(Af, n, n, n).astype(np.float64)
    lu, ipiv, info, out = factor(h, Af, n, n, 32)
    assert info == 0
    assert O.factor_residual(A, lu, ipiv, EPS32) < 16
    b = synth.uniform_pm1(synth.draws(6400, 5, n)).astype(np.float32)
    x = solve(h, out, n, n, ipiv, b)
    assert O.hpl_residual(A, x, b.astype(np.float64), EPS32) < 16


def test_narrow_panels_for_tall_matrices(h):
    """n = 22000: more panel rows than 32-column panels fit in the shared
    memory of a cluster of 16 blocks (21840), so the first block is factored
    as 16-column panels.  Checked by HPL's scaled residual (the O(n^3) factor
    residual is left to the smaller cases)."""
    n = 22000
    Af = synth.uniform_matrix(22000, 0, n, n, n)
    lu, ipiv, info, out = factor(h, Af, n, n, 128)
    assert info == 0
    assert all(j + 1 <= p <= n for j, p in enumerate(ipiv))
    A = synth.logical(Af, n, n, n).astype(np.float64)
    b = synth.uniform_pm1(synth.draws(22000, 5, n)).astype(np.float32)
    x = solve(h, out, n, n, ipiv, b)
    assert O.hpl_residual(A, x, b.astype(np.float64), EPS32) < 16


@pytest.mark.parametrize("n,zc,nb", [(1, 0, 0), (10, 3, 0), (50, 17, 8), (50, 49, 16), (140, 64, 32)])
def test_zero_pivot_info(h, n, zc, nb):
    """A column of exact zeros stays zero through the updates, so step zc
    meets an exactly zero pivot: info = zc + 1, and the factorisation still
    completes, as the oracle's does."""
    A = clear_pivot_matrix(300 + n, n)
    A[:, zc] = 0.0
    lda = n
    lu, ipiv, info, _ = factor(h, colmajor(A, lda), n, lda, nb)
    want, wpiv, zero = O.lu_factor(A.astype(np.float64))
    assert zero == zc and info == zc + 1
    assert np.array_equal(ipiv[:zc], wpiv[:zc])
    assert np.all(lu[zc:, zc] == 0.0)


def test_zero_matrix(h):
    n = 20
    lu, ipiv, info, _ = factor(h, np.zeros(n * n, np.float32), n, n, 8)
    assert info == 1
    assert np.array_equal(ipiv, np.arange(1, n + 1))
    assert np.all(lu == 0.0)


def test_empty(h):
    import torch
    info = torch.full((1,), 5, dtype=torch.int32, device="cuda")
    dA = torch.zeros(1, device="cuda")
    assert h.sgetrf(0, dA, 1, None, info) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert h.sgetrs(0, 1, dA, 1, None, dA, 1) == 0


def test_deterministic(h):
    n = 700
    Af = synth.uniform_matrix(77, 0, n, n, n)
    _, p1, _, o1 = factor(h, Af, n, n)
    _, p2, _, o2 = factor(h, Af, n, n)
    assert np.array_equal(p1, p2)
    assert np.array_equal(o1.view(np.uint32), o2.view(np.uint32))


def test_solve_global_memory_path(h):
    """n > 32768: the solve keeps b in global memory.  Bidiagonal factors
    (L unit lower with one subdiagonal, U upper with one superdiagonal) and
    exchanges with ipiv[j] >= j + 1 give the exact answer by the two
    recurrences y_i = c_i - l_i y_(i-1), x_i = (y_i - u_i x_(i+1)) / d_i."""
    import torch
    n = 32800
    l = 0.5 * synth.uniform_pm1(synth.draws(5, 1, n)).astype(np.float32)
    u = 0.5 * synth.uniform_pm1(synth.draws(5, 2, n)).astype(np.float32)
    d = (1.5 + 0.5 * synth.uniform_pm1(synth.draws(5, 3, n))).astype(np.float32)
    ipiv = (np.arange(n) + 1 + synth.int_range(synth.draws(5, 4, n), 0, 3)).clip(max=n).astype(np.int64)
    b = synth.uniform_pm1(synth.draws(5, 6, n)).astype(np.float32)
    dLU = torch.zeros((n, n), dtype=torch.float32, device="cuda")  # column-major: dLU[j, i] = LU(i, j)
    idx = torch.arange(n, device="cuda")
    dLU[idx, idx] = torch.from_numpy(d).cuda()
    dLU[idx[:-1], idx[1:]] = torch.from_numpy(l[1:]).cuda()   # LU(i, i-1) = l_i (column i-1, row i)
    dLU[idx[1:], idx[:-1]] = torch.from_numpy(u[:-1]).cuda()  # LU(i, i+1) = u_i (column i+1, row i)
    dP = torch.from_numpy(ipiv.astype(np.int32)).cuda()
    db = torch.from_numpy(b).cuda()
    h.sgetrs(n, 1, dLU, n, dP, db, n)
    torch.cuda.synchronize()
    x = db.cpu().numpy().astype(np.float64)
    c = O.apply_pivots(b.astype(np.float64), ipiv)
    y = np.empty(n)
    y[0] = c[0]
    for i in range(1, n):
        y[i] = c[i] - float(l[i]) * y[i - 1]
    want = np.empty(n)
    want[n - 1] = y[n - 1] / float(d[n - 1])
    for i in range(n - 2, -1, -1):
        want[i] = (y[i] - float(u[i]) * want[i + 1]) / float(d[i])
    # each recurrence is contracting (|l|, |u| <= 0.5, d >= 1): errors stay a few eps
    assert np.max(np.abs(x - want)) <= 64 * EPS32 * max(1.0, np.max(np.abs(want)))
