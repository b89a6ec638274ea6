"""GPU parity: the C-ABI sgemm (both paths) against the FP64 CPU oracle.

Pass criterion everywhere: |C_gpu - C64|_ij <= 2 max(k,1) 2^-24 (|alpha| sum|a||b|
+ |beta||c|)_ij (error ratio <= 1), bit-exact for integer-valued inputs, and
no write outside rows 0..m-1 of C (NaN sentinels in the leading-dimension
padding stay intact).
"""

import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

from gpu_util import SIMT, SPLIT, check_full, dev, run_sgemm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    assert torch.cuda.is_available()
    hd = gbgemm.Handle(0)
    hd.set_stream(torch.cuda.current_stream())
    yield hd
    hd.close()


DIMS = [1, 2, 3, 5, 8, 17, 31, 64, 129]
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]
AB = [(1.0, 0.0), (-1.5, 1.0), (1.0, -0.25), (0.0, 0.5), (2.0, 0.0)]


def test_simt_bruteforce_grid(h):
    case = 0
    worst = 0.0
    for m, n, k in itertools.product(DIMS, DIMS, DIMS):
        ta, tb = TRANS[case % 4]
        alpha, beta = AB[case % 5]
        pad = [0, 1, 8][case % 3]
        case += 1
        A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", case, ta, tb, m, n, k, pad=pad)
        worst = max(worst, check_full(h, SIMT, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=4))
    assert worst <= 1.0


@pytest.mark.parametrize("ta,tb", list(itertools.product("NnTtCc", "NnTtCc")))
def test_every_transpose_letter(h, ta, tb):
    m, n, k = 37, 29, 131
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 3, ta, tb, m, n, k, pad=1)
    for path in (SIMT, SPLIT):
        check_full(h, path, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc)


def test_split_grid_guaranteed_k(h):
    case = 0
    for m, n, k in itertools.product([1, 3, 17, 129, 200, 300], [1, 5, 129, 256, 257, 520], [128, 129, 255, 300]):
        ta, tb = TRANS[case % 4]
        alpha, beta = AB[case % 5]
        pad = [0, 1, 8][case % 3]
        case += 1
        A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 100 + case, ta, tb, m, n, k, pad=pad)
        check_full(h, SPLIT, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=4)


def test_split_grid_short_k(h):
    # 16 <= k < 128: the three-part split (six products) drops mid*lo3 + lo3*mid
    # + lo3*lo3 (at most about 2^-23 |a||b| per term) and its FP32 accumulation
    # rounds at most once per 16-deep MMA (6 ceil(k / 16) roundings of at most
    # sum |a||b| 2^-24 each): together below the bound 2 k 2^-24 sum |a||b| from
    # k = 16 on.  (At k = 1 the dropped terms alone can reach the bound.)
    case = 0
    for m, n, k in itertools.product([1, 17, 129, 300], [1, 64, 200, 257], [16, 17, 31, 33, 64, 100, 127]):
        ta, tb = TRANS[case % 4]
        alpha, beta = AB[case % 5]
        pad = [0, 1, 8][case % 3]
        case += 1
        A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 400 + case, ta, tb, m, n, k, pad=pad)
        check_full(h, SPLIT, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=4)


@pytest.mark.parametrize("path", [SIMT, SPLIT])
@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("m,n,k,pad", [(1000, 777, 555, 8), (513, 1030, 1024, 0), (129, 2000, 300, 3)])
def test_multi_tile_ragged(h, path, ta, tb, m, n, k, pad):
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 7, ta, tb, m, n, k, pad=pad)
    check_full(h, path, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc)


def test_plain_256_cube_simt(h):
    # 256^3, N/N, ld 256, alpha 1, beta 0.5, uniform[-1,1] seed 0: the small SIMT case.
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 0, "N", "N", 256, 256, 256)
    check_full(h, SIMT, "N", "N", 256, 256, 256, 1.0, A, lda, B, ldb, 0.5, C, ldc)


@pytest.mark.parametrize("path", [SIMT, SPLIT])
@pytest.mark.parametrize("ta,tb", TRANS)
def test_square_1024_padded(h, path, ta, tb):
    n = 1024
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 1, ta, tb, n, n, n, pad=8)
    check_full(h, path, ta, tb, n, n, n, 1.5, A, lda, B, ldb, -0.25, C, ldc)


@pytest.mark.parametrize("path", [SIMT, SPLIT])
@pytest.mark.parametrize("k", [1, 5, 31, 64, 200, 1000])
def test_small_integers_bit_exact(h, path, k):
    m, n = 300, 270
    for ta, tb in TRANS:
        A, lda, B, ldb, C, ldc = synth.gemm_problem("smallint", 11, ta, tb, m, n, k, pad=2)
        out = run_sgemm(h, path, ta, tb, m, n, k, 2.0, A, lda, B, ldb, -3.0, C, ldc)
        c64, _ = O.gemm_f64(ta, tb, m, n, k, 2.0, A, lda, B, ldb, -3.0, C, ldc)
        assert np.array_equal(synth.logical(out, m, n, ldc).astype(np.float64), c64)
        assert synth.padding_is_sentinel(out, m, n, ldc)


@pytest.mark.parametrize("path", [SIMT, SPLIT])
@pytest.mark.parametrize("k", [1, 128, 4097])
def test_all_ones_equals_k(h, path, k):
    m, n = 130, 260
    A = np.ones(m * k, dtype=np.float32)
    B = np.ones(k * n, dtype=np.float32)
    C = np.full(m * n, np.nan, dtype=np.float32)
    out = run_sgemm(h, path, "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m)
    assert np.all(out == k)


@pytest.mark.parametrize("path", [SIMT, SPLIT])
def test_identity_and_permutation(h, path):
    m, k = 300, 256
    n = k
    A = synth.uniform_matrix(4, 0, m, k, m)
    C = synth.uniform_matrix(4, 4, m, n, m)
    eye = np.eye(k, dtype=np.float32)
    check_full(h, path, "N", "N", m, n, k, -1.5, A, m, eye.reshape(-1), k, 0.5, C, m)
    perm = np.random.default_rng(1).permutation(k)
    P = np.zeros((k, n), dtype=np.float32)
    P[perm, np.arange(n)] = 1.0
    Pcm = P.T.reshape(-1)  # column-major k x n
    check_full(h, path, "N", "N", m, n, k, 1.0, A, m, Pcm, k, 0.0, C, m)
    if path == SIMT:
        # one exact product per entry: the SIMT path reproduces A's columns bit for bit
        out = run_sgemm(h, path, "N", "N", m, n, k, 1.0, A, m, Pcm, k, 0.0, C, m)
        assert np.array_equal(synth.logical(out, m, n, m), synth.logical(A, m, k, m)[:, perm])


@pytest.mark.parametrize("path", [SIMT, SPLIT])
def test_rank1_products(h, path):
    m, n = 200, 300
    for k in ([1] if path == SIMT else []) + [256]:
        A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 12, "N", "T", m, n, k)
        check_full(h, path, "N", "T", m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc)


@pytest.mark.parametrize("path", [SIMT, SPLIT])
def test_blas_conventions(h, path):
    m, n, k = 150, 140, 256
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 13, "N", "N", m, n, k, pad=4)
    Cnan = C.copy()
    Cnan[:] = np.nan
    # beta == 0: C is not read, NaN does not propagate
    out = run_sgemm(h, path, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, Cnan, ldc)
    assert np.all(np.isfinite(synth.logical(out, m, n, ldc)))
    # alpha == 0: A and B are not read (null pointers) and C := beta*C
    out = run_sgemm(h, path, "N", "N", m, n, k, 0.0, None, lda, None, ldb, -0.25, C, ldc, null_ab=True)
    assert np.array_equal(synth.logical(out, m, n, ldc), np.float32(-0.25) * synth.logical(C, m, n, ldc))
    assert synth.padding_is_sentinel(out, m, n, ldc)
    out = run_sgemm(h, path, "N", "N", m, n, k, 0.0, None, lda, None, ldb, 0.0, Cnan, ldc, null_ab=True)
    assert np.all(synth.logical(out, m, n, ldc) == 0.0)
    # k == 0: C := beta*C
    out = run_sgemm(h, path, "N", "N", m, n, 0, 1.0, A, lda, B, 1, 2.0, C, ldc)
    assert np.array_equal(synth.logical(out, m, n, ldc), np.float32(2.0) * synth.logical(C, m, n, ldc))
    # alpha == 0 and beta == 1: quick return, C untouched bit for bit
    out = run_sgemm(h, path, "N", "N", m, n, k, 0.0, A, lda, B, ldb, 1.0, Cnan, ldc)
    assert np.array_equal(out.view(np.uint32), Cnan.view(np.uint32))
    assert h.last_path() == 0
    # m == 0 / n == 0: nothing touched
    for mm, nn in ((0, n), (m, 0)):
        out = run_sgemm(h, path, "N", "N", mm, nn, k, 1.0, A, max(1, mm), B, ldb, 0.0, C, max(1, mm))
        assert np.array_equal(out.view(np.uint32), C.view(np.uint32))


@pytest.mark.parametrize("path", [SIMT, SPLIT])
def test_nonfinite_positions(h, path):
    m, n, k = 64, 96, 256
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 14, "N", "N", m, n, k)
    A = A.copy()
    A[5 + 7 * lda] = np.inf       # row 5 of op(A)
    A[9 + 3 * lda] = np.nan       # row 9
    out = run_sgemm(h, path, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc)
    c64, _ = O.gemm_f64("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc)
    got = synth.logical(out, m, n, ldc)
    assert np.array_equal(~np.isfinite(got), ~np.isfinite(c64))
    if path == SIMT:
        assert np.array_equal(np.isnan(got), np.isnan(c64))
        assert np.array_equal(np.isposinf(got), np.isposinf(c64))


def test_split_extreme_scaling(h):
    # Rows of op(A) scaled by 2^e_i with e_i in [-100, 100] and columns of op(B)
    # by 2^f_j with f_j in [-20, 20]: every product stays in the normal range,
    # but unscaled BF16 parts would leave it (lo underflows near 2^-100 rows).
    m, n, k = 256, 256, 512
    rng_e = synth.int_range(synth.draws(5, 70, m), -100, 100)
    rng_f = synth.int_range(synth.draws(5, 71, n), -20, 20)
    Al = synth.logical(synth.uniform_matrix(5, 0, m, k, m), m, k, m).astype(np.float64)
    Bl = synth.logical(synth.uniform_matrix(5, 2, k, n, k), k, n, k).astype(np.float64)
    Al = (Al * np.ldexp(1.0, rng_e)[:, None]).astype(np.float32)
    Bl = (Bl * np.ldexp(1.0, rng_f)[None, :]).astype(np.float32)
    A = np.ascontiguousarray(Al.T).reshape(-1)
    B = np.ascontiguousarray(Bl.T).reshape(-1)
    C = synth.uniform_matrix(5, 4, m, n, m)
    check_full(h, SPLIT, "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m)
    # Near the top of the range: every entry of op(A) within 0.4% of FLT_MAX,
    # many above 2^128 (1 - 2^-9) where an unscaled BF16 hi rounds to Inf;
    # op(B) entries near 2^-100 keep the products ordinary.
    u = synth.uniform_pm1(synth.draws(5, 72, m * k)).astype(np.float64)
    A2 = np.minimum(3.39e38 + np.abs(u) * 0.0128e38, 3.4028234e38) * np.sign(u + 0.25)
    A2 = A2.astype(np.float32)
    B2 = (synth.uniform_matrix(5, 74, k, n, k).astype(np.float64) * 2.0**-100).astype(np.float32)
    assert np.abs(A2).max() > 3.3961e38
    check_full(h, SPLIT, "N", "N", m, n, k, 1.0, A2, m, B2, k, 0.0, C, m)
    check_full(h, SIMT, "N", "N", m, n, k, 1.0, A2, m, B2, k, 0.0, C, m)


def unpack_panel(panel: np.ndarray, rows: int, k: int):
    RB = (rows + 255) // 256 * 2
    KC = (k + 31) // 32
    P = panel.view(np.uint16).reshape(KC, RB, 128, 8, 8)  # [kc][rb][row][chunk position][element]
    r = np.arange(128)[:, None]
    pos = np.arange(8)[None, :] ^ (r & 7)
    L = P[:, :, r, pos, :]                                  # [kc][rb][row][logical chunk][element]
    hi = L[:, :, :, 0:4, :].reshape(KC, RB, 128, 32).transpose(1, 2, 0, 3).reshape(RB * 128, KC * 32)
    lo = L[:, :, :, 4:8, :].reshape(KC, RB, 128, 32).transpose(1, 2, 0, 3).reshape(RB * 128, KC * 32)
    return hi, lo


def unpack_compact_lo3(panel2: np.ndarray, rows: int, k: int):
    """lo3 (rows padded as in the panel) x (k chunks of 32): block (j, rb) holds
    k chunk 2j in logical chunks 0-3 and chunk 2j+1 in 4-7."""
    RB = (rows + 255) // 256 * 2
    KC = (k + 31) // 32
    KP = (KC + 1) // 2
    P = panel2[: KP * RB * 16384].view(np.uint16).reshape(KP, RB, 128, 8, 8)
    r = np.arange(128)[:, None]
    pos = np.arange(8)[None, :] ^ (r & 7)
    L = P[:, :, r, pos, :]                                  # [pair][rb][row][logical chunk][element]
    even = L[:, :, :, 0:4, :].reshape(KP, RB, 128, 32)
    odd = L[:, :, :, 4:8, :].reshape(KP, RB, 128, 32)
    both = np.stack([even, odd], axis=1).reshape(2 * KP, RB, 128, 32)[:KC]   # [kc][rb][row][32]
    return both.transpose(1, 2, 0, 3).reshape(RB * 128, KC * 32)


@pytest.mark.parametrize("which,trans", [("A", "N"), ("A", "T"), ("B", "N"), ("B", "T")])
@pytest.mark.parametrize("rows,k", [(1, 1), (130, 37), (300, 300), (257, 1000), (200, 600), (70, 160), (90, 480)])
def test_split_pack_bit_exact(h, which, trans, rows, k):
    """The packing launch's panels and row maxima equal the oracle's split bit
    for bit, rows scaled by 2^-60 .. 2^60 so that the re-pack of badly scaled
    rows runs."""
    import torch
    from paper_1608_05265_gb300 import gbgemm
    kcontig = (which == "A") == (trans == "T")
    sr, sc = (k, rows) if kcontig else (rows, k)   # stored shape of X
    ld = sr + 3
    X = synth.normal_rowscaled_matrix(21, 0, sr, sc, ld, elo=-60, ehi=60)
    dX = dev(X)
    amax = torch.zeros(rows, dtype=torch.int32, device="cuda")
    panel = torch.full((gbgemm.panel_bytes(rows, k),), 0x5A, dtype=torch.uint8, device="cuda")
    panel2 = torch.full((gbgemm.panel_bytes(rows, k),), 0x5A, dtype=torch.uint8, device="cuda")
    assert h.split_pack(which, trans, rows, k, dX, ld, amax, panel, panel2) == 0
    torch.cuda.synchronize()
    e, hi, lo, lo3 = O.split_operand3(which, trans, rows, k, X, ld)
    ghi, glo = unpack_panel(panel.cpu().numpy(), rows, k)
    assert np.array_equal(ghi[:rows, :k], hi)
    assert np.array_equal(glo[:rows, :k], lo)
    assert np.all(ghi[rows:] == 0) and np.all(glo[rows:] == 0)
    assert np.all(ghi[:, k:] == 0) and np.all(glo[:, k:] == 0)
    if k < 512:  # three-part split: lo3 in the compact second panel
        KC = (k + 31) // 32
        g3 = unpack_compact_lo3(panel2.cpu().numpy(), rows, k)
        assert np.array_equal(g3[:rows, :k], lo3)
        assert np.all(g3[rows:, :KC * 32] == 0) and np.all(g3[:, k:KC * 32] == 0)
    am = amax.cpu().numpy().view(np.uint32)
    L = synth.logical(X, sr, sc, ld)
    vec = L.T if kcontig else L
    want = np.abs(vec).max(axis=1).astype(np.float32).view(np.uint32)
    assert np.array_equal(am, want)


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("m,n,k,pad", [(1000, 777, 555, 3), (129, 2000, 300, 1), (300, 260, 64, 0), (257, 513, 129, 5)])
def test_odd_leading_dimensions(h, ta, tb, m, n, k, pad):
    """Two-part and three-part splits with odd leading dimensions (rows and
    columns that are not 16-byte aligned) stay within the bound."""
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 17, ta, tb, m, n, k, pad=pad)
    check_full(h, SPLIT, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc, nthreads=4)


@pytest.mark.parametrize("path", [SIMT, SPLIT])
def test_deterministic(h, path):
    m, n, k = 700, 600, 900
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 15, "T", "N", m, n, k)
    o1 = run_sgemm(h, path, "T", "N", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc)
    o2 = run_sgemm(h, path, "T", "N", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc)
    assert np.array_equal(o1.view(np.uint32), o2.view(np.uint32))


def test_auto_path_choice(h):
    from paper_1608_05265_gb300 import gbgemm
    m, n = 100, 100
    for k, want in ((127, gbgemm.PATH_SIMT), (128, gbgemm.PATH_SPLIT_BF16)):
        A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 16, "N", "N", m, n, k)
        check_full(h, gbgemm.PATH_AUTO, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc)
        assert h.last_path() == want

