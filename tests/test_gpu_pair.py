"""Pair tiles on the split path: clusters of two CTAs that compute 256 x 256
tiles with tcgen05 MMAs of cta_group::2 (each CTA loads its own 128-row A
block and half of the tile's B rows).  Calls take them for the widest tiles
(256 columns) with at least two tile rows: with two-part panels (k >= 512),
with or without k slices, and with three-part panels from 8 k chunks.
The schedule is pinned to BN 256 without k slicing so that small ragged
shapes take pair tiles too: an odd number of tile rows (the last pair's
second half lies past m), ragged tile columns, every transpose, badly scaled
rows and columns on either CTA of a pair, beta = 0, k slices and a strided
batch.
Each is checked against the FP64 oracle under the componentwise bound."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

from gpu_util import SPLIT, check_full, dev

pytestmark = pytest.mark.gpu

# schedule 3 + 12 b + 4 r + q: BN 64 << 2 = 256, tile-row groups of 16, no k slicing
PAIR_SCHEDULE = 3 + 12 * 2 + 4 * 2 + 0


@pytest.fixture(scope="module")
def h():
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    hd = gbgemm.Handle(0)
    hd.set_stream(torch.cuda.current_stream())
    info = gbgemm.schedule_info(PAIR_SCHEDULE)
    assert (info["tile_n"], info["raster"], info["level"]) == (256, 16, 0)
    hd.set_schedule(PAIR_SCHEDULE)
    yield hd
    hd.set_schedule(-1)
    hd.close()


@pytest.mark.parametrize("m,n,k,pad", [
    (300, 700, 600, 3),     # 3 tile rows: the second pair's odd half is empty; 188-column last tile
    (129, 513, 1024, 0),    # one pair, one row in its odd half; 1-column last tile
    (1000, 777, 555, 8),    # 8 tile rows, 4 pairs, k not a multiple of 32
    (640, 1030, 2048, 1),   # 5 tile rows, 5 tile columns
    (300, 700, 300, 3),     # three-part panels (k < 512): six products per k step
    (129, 513, 260, 0),     # three-part, k not a multiple of 32, one pair
])
def test_pair_tiles_ragged(h, m, n, k, pad):
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 95, "N", "N", m, n, k, pad=pad)
    assert check_full(h, SPLIT, "N", "N", m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc, nthreads=4) <= 1.0


@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "T"), ("T", "T")])
def test_pair_tiles_transposes(h, ta, tb):
    m, n, k = 520, 600, 768
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 96, ta, tb, m, n, k, pad=5)
    assert check_full(h, SPLIT, ta, tb, m, n, k, -0.75, A, lda, B, ldb, 2.0, C, ldc, nthreads=4) <= 1.0


@pytest.mark.parametrize("m,n,k", [(300, 260, 4096), (129, 300, 8192), (640, 512, 2048)])
def test_pair_tiles_k_sliced(h, m, n, k):
    """Pair items that are k slices of a 256 x 256 tile (split-K at full fill,
    BN 256): each CTA stores its own 128-row partial tile (none for the empty
    odd half of a last pair) and the reduction sums the slices."""
    from paper_1608_05265_gb300 import gbgemm, predictor
    s = 3 + 12 * 2 + 4 * 2 + 3
    assert gbgemm.schedule_info(s)["level"] == 3
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 94, "T", "N", m, n, k, pad=2)
    assert h.schedule_legal(predictor.tuning_problem(("T", "N", m, n, k, 1, 1, 1)), s)
    h.set_schedule(s)
    try:
        assert check_full(h, SPLIT, "T", "N", m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc, nthreads=4) <= 1.0
        assert h.last_schedule() == s
    finally:
        h.set_schedule(PAIR_SCHEDULE)


def test_pair_tiles_badly_scaled_and_beta_zero(h):
    """Row scales 2^+-60 on the rows of op(A) (both halves of every pair) and
    on the columns of op(B) (both CTAs' B halves); beta = 0 never reads C."""
    m, n, k = 384, 512, 1024
    A = synth.normal_rowscaled_matrix(97, 0, m, k, m, elo=-60, ehi=60)
    Bt = synth.normal_rowscaled_matrix(97, 2, n, k, n, elo=-60, ehi=60)  # op(B) = Bt^T: columns scaled
    C = np.full(m * n, np.nan, dtype=np.float32)  # beta = 0: NaNs in C must not reach the result
    assert check_full(h, SPLIT, "N", "T", m, n, k, 1.0, A, m, Bt, n, 0.0, C, m, nthreads=4) <= 1.0


def test_pair_tiles_three_part_badly_scaled(h):
    """k < 512 (three-part panels, the compact lo3 slots relayed as well) with
    rows of op(A) and columns of op(B) scaled by 2^+-60."""
    m, n, k = 384, 512, 300
    A = synth.normal_rowscaled_matrix(93, 0, m, k, m, elo=-60, ehi=60)
    Bt = synth.normal_rowscaled_matrix(93, 2, n, k, n, elo=-60, ehi=60)
    C = synth.uniform_matrix(93, 4, m, n, m)
    assert check_full(h, SPLIT, "N", "T", m, n, k, 1.0, A, m, Bt, n, 0.5, C, m, nthreads=4) <= 1.0


def test_pair_tiles_strided_batch(h):
    """A strided batch of nine problems of 3 tile rows by 3 tile columns
    (batches take the default schedule: 81 tiles of 128 x 256 fill half the
    SMs, so BN 256 without k slices, so pair tiles)."""
    import torch
    m, n, k, batch = 300, 520, 512, 9
    lda, ldb, ldc = m + 2, k + 1, m + 4
    sa, sb, sc = lda * k + 7, ldb * n + 5, ldc * n + 3
    A = synth.uniform_matrix(98, 0, 1, sa * batch, 1).reshape(-1)
    B = synth.uniform_matrix(98, 2, 1, sb * batch, 1).reshape(-1)
    C = synth.uniform_matrix(98, 4, 1, sc * batch, 1).reshape(-1)
    dA, dB, dC = dev(A), dev(B), dev(C)
    h.set_path(SPLIT)
    h.sgemm_strided_batched("N", "N", m, n, k, 1.25, dA, lda, sa, dB, ldb, sb, 0.5, dC, ldc, sc, batch)
    torch.cuda.synchronize()
    assert h.get_device_status() == 0
    out = dC.cpu().numpy()
    for z in range(batch):
        Az, Bz, Cz = A[z * sa:z * sa + lda * k], B[z * sb:z * sb + ldb * n], C[z * sc:z * sc + ldc * n]
        c64, bnd = O.gemm_f64("N", "N", m, n, k, 1.25, Az, lda, Bz, ldb, 0.5, Cz, ldc, nthreads=4)
        got = synth.logical(out[z * sc:z * sc + ldc * n], m, n, ldc)
        assert O.error_ratio(got, c64, bnd) <= 1.0, z


def test_pair_tiles_deterministic(h):
    """Two runs of the same call give the same bits (pairs take tiles in a fixed order)."""
    import torch
    m, n, k = 768, 1024, 1536
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 99, "N", "N", m, n, k, pad=0)
    dA, dB = dev(A), dev(B)
    h.set_path(SPLIT)
    outs = []
    for _ in range(2):
        dC = dev(C)
        h.sgemm("N", "N", m, n, k, 1.0, dA, lda, dB, ldb, 1.0, dC, ldc)
        torch.cuda.synchronize()
        outs.append(dC.cpu().numpy())
    assert h.get_device_status() == 0
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))
