"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* exact rational arithmetic (Python ``fractions``) on tiny shapes, every
  transpose letter and padded leading dimensions (Section III-A problem
  statement: op(), leading dimensions, arbitrary M, N, K);
* closed forms: identity, permutation, all-ones, rank-1 products;
* integer matrices against numpy's int64 matmul (exact);
* the transposition identity (op(A) op(B))^T = op(B)^T op(A)^T;
* the naive FP32 loop inside the acceptance bound of the FP64 result;
* the FLOP convention against the paper's Tables I, II and VII.
"""

import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LETTERS = ["N", "T", "C", "n", "t", "c"]


def is_t(c):
    return c in "TtCc"


def stored(trans, r, c):
    return (c, r) if is_t(trans) else (r, c)


def exact_gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc):
    """C_out and sum |a||b| in exact rationals, straight from the definition."""
    out = {}
    for j in range(n):
        for i in range(m):
            s = Fraction(0)
            sabs = Fraction(0)
            if alpha != 0 and k > 0:
                for p in range(k):
                    a = Fraction(float(A[p + i * lda] if is_t(transa) else A[i + p * lda]))
                    b = Fraction(float(B[j + p * ldb] if is_t(transb) else B[p + j * ldb]))
                    s += a * b
                    sabs += abs(a) * abs(b)
            c = Fraction(float(C[i + j * ldc])) if beta != 0 else Fraction(0)
            val = (Fraction(float(alpha)) * s if (alpha != 0 and k > 0) else 0) + Fraction(float(beta)) * c
            tot = abs(Fraction(float(alpha))) * sabs + abs(Fraction(float(beta))) * abs(c)
            out[(i, j)] = (val, tot)
    return out


def test_bruteforce_exact_rational_all_letters():
    shapes = list(itertools.product([0, 1, 3, 5], repeat=3))
    alphas = [1.0, -1.5, 0.0]
    betas = [0.0, 1.0, -0.25]
    case = 0
    for (m, n, k) in shapes:
        for ta, tb in itertools.product(LETTERS, LETTERS):
            pad = case % 3  # tight, +1, +2
            alpha = alphas[case % 3]
            beta = betas[(case // 3) % 3]
            case += 1
            ar, ac = stored(ta, m, k)
            br, bc = stored(tb, k, n)
            lda, ldb, ldc = max(1, ar + pad), max(1, br + pad), max(1, m + pad)
            A = synth.uniform_matrix(case, 0, ar, ac, lda)
            B = synth.uniform_matrix(case, 2, br, bc, ldb)
            C = synth.uniform_matrix(case, 4, m, n, ldc)
            if m == 0 or n == 0:
                continue
            out, bnd = O.gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
            ex = exact_gemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
            for (i, j), (val, tot) in ex.items():
                allow = (k + 2) * 2.0**-52 * float(tot)
                assert abs(Fraction(out[i, j]) - val) <= Fraction(allow), (ta, tb, m, n, k, i, j)
                want_bnd = 2.0 * max(k, 1) * 2.0**-24 * float(tot)
                assert bnd[i, j] == pytest.approx(want_bnd, rel=1e-12, abs=0.0)


def test_beta_zero_does_not_read_c_and_alpha_zero_does_not_read_ab():
    m, n, k = 4, 3, 5
    A = np.full(m * k, np.nan, dtype=np.float32)
    B = np.full(k * n, np.nan, dtype=np.float32)
    C = synth.uniform_matrix(7, 4, m, n, m)
    out, bnd = O.gemm_f64("N", "N", m, n, k, 0.0, A, m, B, k, 2.0, C, m)
    assert np.array_equal(out, 2.0 * synth.logical(C, m, n, m).astype(np.float64))
    Cn = np.full(m * n, np.nan, dtype=np.float32)
    A = synth.uniform_matrix(7, 0, m, k, m)
    B = synth.uniform_matrix(7, 2, k, n, k)
    out, _ = O.gemm_f64("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, Cn, m)
    assert np.all(np.isfinite(out))
    out32 = O.gemm_f32("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, Cn, m)
    assert np.all(np.isfinite(out32))


@pytest.mark.parametrize("ta", ["N", "T"])
def test_identity_closed_form(ta):
    m, k = 37, 29
    n = k
    alpha, beta = -1.5, 0.5
    ar, ac = stored(ta, m, k)
    A = synth.uniform_matrix(1, 0, ar, ac, ar + 3)
    Bm = np.eye(k, dtype=np.float32)
    B = synth.place_colmajor(Bm.T.reshape(-1), k, n, k + 1)
    C = synth.uniform_matrix(1, 4, m, n, m + 2)
    out, _ = O.gemm_f64(ta, "N", m, n, k, alpha, A, ar + 3, B, k + 1, beta, C, m + 2)
    opA = synth.logical(A, ar, ac, ar + 3).astype(np.float64)
    opA = opA.T if ta == "T" else opA
    want = alpha * opA + beta * synth.logical(C, m, n, m + 2).astype(np.float64)
    assert np.array_equal(out, want)


def test_permutation_closed_form():
    m, k = 23, 17
    n = k
    perm = np.random.default_rng(0).permutation(k)
    Pm = np.zeros((k, n), dtype=np.float32)
    Pm[perm, np.arange(n)] = 1.0  # column j of op(B) selects column perm[j] of op(A)
    A = synth.uniform_matrix(2, 0, m, k, m)
    # op(B) = Pm with transb = T: store Pm^T (n x k) column-major.
    B = synth.place_colmajor(Pm.reshape(-1), n, k, n)
    C = synth.uniform_matrix(2, 4, m, n, m)
    out, _ = O.gemm_f64("N", "T", m, n, k, 1.0, A, m, B, n, 0.0, C, m)
    opA = synth.logical(A, m, k, m).astype(np.float64)
    assert np.array_equal(out, opA[:, perm])


@pytest.mark.parametrize("k", [1, 7, 256, 1000])
def test_all_ones_equals_k(k):
    m, n = 9, 11
    A = np.ones(m * k, dtype=np.float32)
    B = np.ones(k * n, dtype=np.float32)
    C = np.ones(m * n, dtype=np.float32)
    out, _ = O.gemm_f64("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m)
    assert np.all(out == k)
    out, _ = O.gemm_f64("T", "T", m, n, k, 1.0, A, k, B, n, 1.0, C, m)
    assert np.all(out == k + 1)
    assert np.all(O.gemm_f32("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m) == k)


def test_rank1_closed_form():
    m, n = 13, 19
    A = synth.uniform_matrix(3, 0, m, 1, m)
    B = synth.uniform_matrix(3, 2, 1, n, 1)
    C = synth.uniform_matrix(3, 4, m, n, m)
    alpha, beta = 1.5, -0.25
    out, _ = O.gemm_f64("N", "N", m, n, 1, alpha, A, m, B, 1, beta, C, m)
    a = A[:m].astype(np.float64)
    b = B[:n].astype(np.float64)
    want = alpha * (a[:, None] * b[None, :]) + beta * synth.logical(C, m, n, m).astype(np.float64)
    assert np.array_equal(out, want)
    # rank-1 matrix u v^T with large k: sum_p u_i w_p w_p v_j = u_i v_j sum w_p^2.
    k = 333
    w = synth.small_int_matrix(3, 6, k, 1, k)[:k]
    u = synth.small_int_matrix(3, 8, m, 1, m)[:m]
    v = synth.small_int_matrix(3, 10, n, 1, n)[:n]
    A2 = (u[:, None] * w[None, :]).T.reshape(-1).astype(np.float32)   # m x k column-major
    B2 = (w[:, None] * v[None, :]).T.reshape(-1).astype(np.float32)   # k x n column-major
    out, _ = O.gemm_f64("N", "N", m, n, k, 1.0, A2, m, B2, k, 0.0, C, m)
    want = np.outer(u.astype(np.float64), v.astype(np.float64)) * float(np.sum(w.astype(np.float64) ** 2))
    assert np.array_equal(out, want)


@pytest.mark.parametrize("ta,tb", list(itertools.product(LETTERS, LETTERS)))
def test_small_integers_exact(ta, tb):
    m, n, k = 21, 14, 45
    A, lda, B, ldb, C, ldc = synth.gemm_problem("smallint", 5, ta, tb, m, n, k, pad=3)
    alpha, beta = 2.0, -3.0
    out, _ = O.gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
    out32 = O.gemm_f32(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
    ar, ac = stored(ta, m, k)
    br, bc = stored(tb, k, n)
    Ai = synth.logical(A, ar, ac, lda).astype(np.int64)
    Bi = synth.logical(B, br, bc, ldb).astype(np.int64)
    Ci = synth.logical(C, m, n, ldc).astype(np.int64)
    opA = Ai.T if is_t(ta) else Ai
    opB = Bi.T if is_t(tb) else Bi
    want = 2 * (opA @ opB) - 3 * Ci
    assert np.array_equal(out, want.astype(np.float64))
    assert np.array_equal(out32.astype(np.float64), want.astype(np.float64))


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
def test_transposition_identity(ta, tb):
    m, n, k = 17, 23, 31
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 6, ta, tb, m, n, k, pad=1)
    out, _ = O.gemm_f64(ta, tb, m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc)
    flip = {"N": "T", "T": "N"}
    C2 = np.zeros(n * m, dtype=np.float32)
    out2, _ = O.gemm_f64(flip[tb], flip[ta], n, m, k, 1.0, B, ldb, A, lda, 0.0, C2, n)
    assert np.array_equal(out, out2.T)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
def test_fp32_variant_within_bound(ta, tb):
    m, n, k = 40, 33, 300
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 8, ta, tb, m, n, k, pad=8)
    out, bnd = O.gemm_f64(ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc)
    out32 = O.gemm_f32(ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc)
    r = O.error_ratio(out32, out, bnd)
    assert r <= 1.0
    assert r > 0.0  # the naive loop does round


def test_block_matches_full():
    m, n, k = 50, 41, 60
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 9, "T", "N", m, n, k, pad=2)
    full, fb = O.gemm_f64("T", "N", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc)
    blk, bb = O.gemm_f64("T", "N", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc, rows=(7, 30), cols=(5, 41), nthreads=3)
    assert np.array_equal(blk, full[7:30, 5:41])
    assert np.array_equal(bb, fb[7:30, 5:41])


def test_freivalds_accepts_oracle_and_rejects_planted_error():
    m, n, k = 64, 48, 200
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 10, "N", "T", m, n, k)
    out, _ = O.gemm_f64("N", "T", m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc)
    opA = synth.logical(A, m, k, lda)
    opB = synth.logical(B, n, k, ldb).T
    Cin = synth.logical(C, m, n, ldc)
    x = np.where(synth.draws(1, 0, n) >> np.uint64(63), 1.0, -1.0)
    good = out.astype(np.float32)
    assert O.freivalds_ratio(opA, opB, Cin, good, 1.5, -0.25, x) <= 1.0
    bad = good.copy()
    bad[5, 7] += 0.5  # far above the row allowance (about 2*200*2^-24*sum|a||b| ~ 1e-3)
    assert O.freivalds_ratio(opA, opB, Cin, bad, 1.5, -0.25, x) > 1.0


def test_error_ratio_zero_bound_requires_exact():
    c64 = np.array([[1.0, 0.0]])
    bnd = np.array([[1e-6, 0.0]])
    assert O.error_ratio(np.array([[1.0, 0.0]], dtype=np.float32), c64, bnd) == 0.0
    assert O.error_ratio(np.array([[1.0, 1e-30]], dtype=np.float32), c64, bnd) == math.inf


def test_flop_convention_matches_paper_tables():
    from paper_1608_05265_gb300.metrics import gemm_flops
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_table1_flops.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for r in rows:
        m, n, k, t, g = int(r[0]), int(r[1]), int(r[2]), float(r[3]), float(r[4])
        assert round(gemm_flops(m, n, k) / t / 1e9, 3) == pytest.approx(g, abs=1.5e-3)
    N, t, g, scaled, res = [l.split() for l in open(os.path.join(GOLDEN, "paper_hpl.txt")) if not l.startswith("#")][0]
    N, t, g, scaled, res = int(N), float(t), float(g), float(scaled), float(res)
    hpl_flops = 2.0 / 3.0 * N**3 + 2.0 * N**2
    assert round(hpl_flops / t / 1e9, 3) == pytest.approx(g, abs=1e-3)
    assert scaled * 2.0**-53 == pytest.approx(res, rel=2e-3)
