"""CPU models of the schedules the GPU LU runs, checked against the FP64
oracle (partial pivoting, the paper's HPL factorisation, Section IV-C).

They pin the decomposition, not the kernels: that factoring a panel as
slabs of rows whose blocks exchange only their candidates, and that the
blocked factorisation in the order its two streams run it (look-ahead, and
the single-panel variant whose next panel applies the previous block to its
own columns), give exactly the pivots and factors of unblocked partial
pivoting.  The models use float64 numpy and no library code.
"""

import numpy as np
import pytest

from oracle import lu_ref as O


def panel_by_slabs(A, C):
    """Partial pivoting of a tall R x w panel held as C slabs of rows: per
    column each slab proposes its largest |a| below the diagonal (first row
    on ties), every slab picks the same winner (largest value, smallest row),
    the pivot row and row q trade places, and every slab updates its rows."""
    R, w = A.shape
    RS = -(-R // C)
    slabs = [A[c * RS:min(R, (c + 1) * RS)].copy() for c in range(C)]
    piv = []
    for q in range(w):
        cands = []
        for c in range(C):
            best, bi = -1.0, None
            for rr in range(len(slabs[c])):
                r = c * RS + rr
                if r >= q and abs(slabs[c][rr, q]) > best:
                    best, bi = abs(slabs[c][rr, q]), r
            cands.append((best, bi))
        p, top = q, (-1.0, None)
        for v, i in cands:
            if i is not None and (top[1] is None or v > top[0] or (v == top[0] and i < top[1])):
                top = (v, i)
        if top[1] is not None:
            p = top[1]
        oq, op = q // RS, p // RS
        prow = slabs[op][p - op * RS].copy()
        qrow = slabs[oq][q - oq * RS].copy()
        slabs[oq][q - oq * RS] = prow
        slabs[op][p - op * RS] = qrow
        piv.append(p + 1)
        if prow[q] != 0:
            for c in range(C):
                for rr in range(len(slabs[c])):
                    if c * RS + rr > q:
                        slabs[c][rr, q] /= prow[q]
                        slabs[c][rr, q + 1:] -= slabs[c][rr, q] * prow[q + 1:]
    return np.vstack(slabs), piv


def unblocked_panel(A):
    lu = A.copy()
    piv = []
    for j in range(A.shape[1]):
        p = j + int(np.argmax(np.abs(lu[j:, j])))
        piv.append(p + 1)
        lu[[j, p]] = lu[[p, j]]
        if lu[j, j] != 0:
            lu[j + 1:, j] /= lu[j, j]
            lu[j + 1:, j + 1:] -= np.outer(lu[j + 1:, j], lu[j, j + 1:])
    return lu, piv


@pytest.mark.parametrize("R,w,C", [(1, 1, 1), (37, 5, 3), (130, 32, 8), (300, 13, 16), (64, 32, 8)])
def test_panel_exchange_equals_partial_pivoting(R, w, C):
    rng = np.random.default_rng(R + w + C)
    A = rng.uniform(-1, 1, (R, w))
    if R > 3:
        A[:, min(2, w - 1)] = 0.0  # a zero pivot on the way
    got, piv = panel_by_slabs(A, C)
    want, wpiv = unblocked_panel(A)
    assert piv == wpiv
    assert np.allclose(got, want, rtol=0, atol=1e-12)


class Blocked:
    """The blocked factorisation as the library's streams run it."""

    def __init__(self, A):
        self.A = A.copy()
        self.n = A.shape[0]
        self.ipiv = np.zeros(self.n, dtype=np.int64)

    def panel(self, j1, w):  # rows [j1, n) x columns [j1, j1 + w)
        A = self.A
        for q in range(w):
            c = j1 + q
            p = c + int(np.argmax(np.abs(A[c:, c])))
            self.ipiv[c] = p + 1
            A[[c, p], j1:j1 + w] = A[[p, c], j1:j1 + w]
            if A[c, c] != 0:
                A[c + 1:, c] /= A[c, c]
                A[c + 1:, c + 1:j1 + w] -= np.outer(A[c + 1:, c], A[c, c + 1:j1 + w])

    def exchange(self, j1, w, cols):
        for q in range(w):
            r, p = j1 + q, self.ipiv[j1 + q] - 1
            if p != r:
                self.A[np.ix_([r, p], cols)] = self.A[np.ix_([p, r], cols)]

    def swap_trsm(self, j1, w, c_lo, r_lo, c_hi):  # columns [c_lo, j1) and [r_lo, c_hi)
        if c_lo < j1:
            self.exchange(j1, w, np.arange(c_lo, j1))
        if r_lo < c_hi:
            self.exchange(j1, w, np.arange(r_lo, c_hi))
            L = np.tril(self.A[j1:j1 + w, j1:j1 + w], -1) + np.eye(w)
            self.A[j1:j1 + w, r_lo:c_hi] = np.linalg.solve(L, self.A[j1:j1 + w, r_lo:c_hi])

    def update(self, r, c, cols, kc, k):
        A = self.A
        A[r:, c:c + cols] -= A[r:, kc:kc + k] @ A[kc:kc + k, c:c + cols]


def factor_lookahead(A, b, pw):
    """Blocks of b columns as panels of pw; after block k's exchanges and U12
    the next block's columns are updated, the next block is factored (side
    stream) and the rest of the trailing matrix updated (main stream)."""
    M = Blocked(A)
    n = M.n

    def factor_block(j0, nbo):
        for j1 in range(j0, j0 + nbo, pw):
            w = min(pw, j0 + nbo - j1)
            M.panel(j1, w)
            if w == nbo:
                return
            M.swap_trsm(j1, w, j0, j1 + w, j0 + nbo)
            cols = j0 + nbo - j1 - w
            if cols > 0:
                M.update(j1 + w, j1 + w, cols, j1, w)

    nbo = min(n, b)
    factor_block(0, nbo)
    j0 = 0
    while j0 < n:
        nbo = min(n - j0, b)
        if j0 > 0 or j0 + nbo < n:
            M.swap_trsm(j0, nbo, 0, j0 + nbo, n)
        jn = j0 + nbo
        if jn >= n:
            break
        nbn = min(n - jn, b)
        M.update(jn, jn, nbn, j0, nbo)
        factor_block(jn, nbn)
        if n - jn - nbn > 0:
            M.update(jn, jn + nbn, n - jn - nbn, j0, nbo)
        j0 = jn
    return M.A, M.ipiv


def factor_fused(A, b):
    """Every block one panel of b columns: the next panel first applies block
    k to its own columns (exchanges, U12, update), while the main stream
    applies block k to every other column."""
    M = Blocked(A)
    n = M.n
    nbo = min(n, b)
    M.panel(0, nbo)
    j0 = 0
    while j0 < n:
        nbo = min(n - j0, b)
        jn = j0 + nbo
        nbn = min(n - jn, b) if jn < n else 0
        if nbn > 0:  # side stream: prologue, then the panel
            M.swap_trsm(j0, nbo, jn, jn, jn + nbn)
            M.update(jn, jn, nbn, j0, nbo)
            M.panel(jn, nbn)
        if j0 > 0 or jn + nbn < n:  # main stream: block k on every other column
            M.swap_trsm(j0, nbo, 0, jn + nbn, n)
        if nbn > 0 and n - jn - nbn > 0:
            M.update(jn, jn + nbn, n - jn - nbn, j0, nbo)
        j0 = jn
    return M.A, M.ipiv


@pytest.mark.parametrize("n,b,pw", [(1, 32, 32), (40, 8, 8), (100, 32, 32), (130, 128, 32), (257, 64, 32),
                                    (300, 13, 13), (333, 128, 16)])
def test_lookahead_schedule_equals_partial_pivoting(n, b, pw):
    A = np.random.default_rng(n + b).uniform(-1, 1, (n, n))
    got, piv = factor_lookahead(A, b, pw)
    want, wpiv, _ = O.lu_factor(A)
    assert np.array_equal(piv, wpiv)
    assert np.allclose(got, want, rtol=0, atol=1e-9)


@pytest.mark.parametrize("n,b", [(1, 32), (5, 32), (64, 32), (100, 32), (257, 32), (300, 13), (200, 1)])
def test_fused_schedule_equals_partial_pivoting(n, b):
    A = np.random.default_rng(3 * n + b).uniform(-1, 1, (n, n))
    got, piv = factor_fused(A, b)
    want, wpiv, _ = O.lu_factor(A)
    assert np.array_equal(piv, wpiv)
    assert np.allclose(got, want, rtol=0, atol=1e-9)
