"""Full-size parity: the FP64 GPU checker against the CPU oracle, then the
square 8192^3 sweep point and the Linpack-shaped trailing updates at the
sizes the benchmark runs, checked on sampled blocks (GPU FP64 checker and CPU
oracle) and by the Freivalds identity."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

from gpu_util import SIMT, SPLIT, dev, freivalds, sample_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    hd = gbgemm.Handle(0)
    hd.set_stream(torch.cuda.current_stream())
    yield hd
    hd.close()


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_gpu_checker_matches_cpu_oracle(h, ta, tb):
    import torch
    m, n, k = 300, 260, 777
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 71, ta, tb, m, n, k, pad=5)
    for path in (SIMT, SPLIT):
        dA, dB, dC, dC0 = dev(A), dev(B), dev(C), dev(C)
        h.set_path(path)
        h.sgemm(ta, tb, m, n, k, 1.5, dA, lda, dB, ldb, -0.25, dC, ldc)
        torch.cuda.synchronize()
        out = dC.cpu().numpy()
        c64, bnd = O.gemm_f64(ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc)
        cpu = O.error_ratio(synth.logical(out, m, n, ldc), c64, bnd)
        gpu = h.check_error(ta, tb, m, n, k, 1.5, dA, lda, dB, ldb, -0.25, dC0, dC, ldc)
        assert gpu == pytest.approx(cpu, rel=1e-9, abs=0.0)
        assert 0.0 < gpu <= 1.0
        blk = h.check_error(ta, tb, m, n, k, 1.5, dA, lda, dB, ldb, -0.25, dC0, dC, ldc, rows=(10, 90), cols=(200, 260))
        cb = O.error_ratio(synth.logical(out, m, n, ldc)[10:90, 200:260], c64[10:90, 200:260], bnd[10:90, 200:260])
        assert blk == pytest.approx(cb, rel=1e-9, abs=0.0)
        # an error of four times the bound in one element is reported
        i, j = 123, 45
        bad = dC.clone()
        bad[i + j * ldc] += float(4.0 * bnd[i, j])
        assert h.check_error(ta, tb, m, n, k, 1.5, dA, lda, dB, ldb, -0.25, dC0, bad, ldc) > 3.0
        bad[i + j * ldc] = float("nan")
        assert h.check_error(ta, tb, m, n, k, 1.5, dA, lda, dB, ldb, -0.25, dC0, bad, ldc) == float("inf")


@pytest.mark.parametrize("path,ta,tb", [(SPLIT, "N", "N"), (SPLIT, "T", "T"), (SPLIT, "T", "N"), (SIMT, "N", "N")])
def test_square_8192(h, path, ta, tb):
    """The square sweep's 8192^3 point: ld = rows + 8, alpha 1.5, beta -0.25, uniform, seed 1."""
    import torch
    n = 8192
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 1, ta, tb, n, n, n, pad=8)
    dA, dB, dC, dC0 = dev(A), dev(B), dev(C), dev(C)
    h.set_path(path)
    h.sgemm(ta, tb, n, n, n, 1.5, dA, lda, dB, ldb, -0.25, dC, ldc)
    torch.cuda.synchronize()
    assert h.get_device_status() == 0
    worst = 0.0
    for rows, cols in sample_blocks(n, n, 512, seed=3, count=2):
        worst = max(worst, h.check_error(ta, tb, n, n, n, 1.5, dA, lda, dB, ldb, -0.25, dC0, dC, ldc, rows, cols))
    assert worst <= 1.0
    out = dC.cpu().numpy()
    assert synth.padding_is_sentinel(out, n, n, ldc)
    rows, cols = (n - 128, n), (4000, 4128)
    c64, bnd = O.gemm_f64(ta, tb, n, n, n, 1.5, A, lda, B, ldb, -0.25, C, ldc, rows=rows, cols=cols)
    cpu = O.error_ratio(synth.logical(out, n, n, ldc)[rows[0]:rows[1], cols[0]:cols[1]], c64, bnd)
    gpu = h.check_error(ta, tb, n, n, n, 1.5, dA, lda, dB, ldb, -0.25, dC0, dC, ldc, rows, cols)
    assert cpu <= 1.0 and gpu == pytest.approx(cpu, rel=1e-9, abs=0.0)
    assert freivalds(out, ta, tb, n, n, n, 1.5, A, lda, B, ldb, -0.25, C, ldc, seed=5) <= 1.0


@pytest.mark.parametrize("mn,nb", [(4096, 128), (4096, 256), (8192, 256)])
def test_linpack_trailing_update(h, mn, nb):
    """C := C - A B with A m x nb, B nb x n, entries normal(0,1) * 2^e per stored
    row, e uniform in [-20, 20] (seed 2), tight leading dimensions."""
    import torch
    m = n = mn
    A = synth.normal_rowscaled_matrix(2, 0, m, nb, m)
    B = synth.normal_rowscaled_matrix(2, 2, nb, n, nb)
    C = synth.normal_rowscaled_matrix(2, 4, m, n, m)
    dA, dB, dC, dC0 = dev(A), dev(B), dev(C), dev(C)
    h.set_path(0)  # AUTO: k = nb >= 128 runs the split path
    h.sgemm("N", "N", m, n, nb, -1.0, dA, m, dB, nb, 1.0, dC, m)
    torch.cuda.synchronize()
    assert h.last_path() == SPLIT and h.get_device_status() == 0
    if mn <= 4096:
        assert h.check_error("N", "N", m, n, nb, -1.0, dA, m, dB, nb, 1.0, dC0, dC, m) <= 1.0
    else:
        for rows, cols in sample_blocks(m, n, 1024, seed=4, count=3):
            assert h.check_error("N", "N", m, n, nb, -1.0, dA, m, dB, nb, 1.0, dC0, dC, m, rows, cols) <= 1.0
    out = dC.cpu().numpy()
    rows, cols = (100, 228), (m - 200, m - 72)
    c64, bnd = O.gemm_f64("N", "N", m, n, nb, -1.0, A, m, B, nb, 1.0, C, m, rows=rows, cols=cols)
    assert O.error_ratio(synth.logical(out, m, n, m)[rows[0]:rows[1], cols[0]:cols[1]], c64, bnd) <= 1.0
    assert freivalds(out, "N", "N", m, n, nb, -1.0, A, m, B, nb, 1.0, C, m, seed=6) <= 1.0


_SQUARE_CACHE = {}


def _square_inputs(n):
    """The square sweep's inputs at size n (seed 1, ld = n + 8): the stored
    shapes are n x n whatever the transposes, so one set serves all four."""
    if n not in _SQUARE_CACHE:
        _SQUARE_CACHE[n] = synth.gemm_problem("uniform", 1, "N", "N", n, n, n, pad=8)
    return _SQUARE_CACHE[n]


@pytest.mark.parametrize("n", [2048, 4096])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("path", [SPLIT, SIMT])
def test_square_sweep_against_cpu_oracle(h, n, ta, tb, path):
    """The square sweep's 2048^3 and 4096^3 points on both paths, against the CPU
    oracle: every element at 2048, sampled 256 x 256 blocks (corners, centre and
    seeded random ones) plus the Freivalds identity at 4096."""
    import torch
    A, lda, B, ldb, C, ldc = _square_inputs(n)
    dA, dB, dC = dev(A), dev(B), dev(C)
    h.set_path(path)
    h.sgemm(ta, tb, n, n, n, 1.5, dA, lda, dB, ldb, -0.25, dC, ldc)
    torch.cuda.synchronize()
    assert h.last_path() == path and h.get_device_status() == 0
    out = dC.cpu().numpy()
    del dA, dB, dC
    assert synth.padding_is_sentinel(out, n, n, ldc)
    got = synth.logical(out, n, n, ldc)
    if n <= 2048:
        c64, bnd = O.gemm_f64(ta, tb, n, n, n, 1.5, A, lda, B, ldb, -0.25, C, ldc)
        assert O.error_ratio(got, c64, bnd) <= 1.0
    else:
        for rows, cols in sample_blocks(n, n, 256, seed=7, count=2):
            c64, bnd = O.gemm_f64(ta, tb, n, n, n, 1.5, A, lda, B, ldb, -0.25, C, ldc, rows=rows, cols=cols)
            assert O.error_ratio(got[rows[0]:rows[1], cols[0]:cols[1]], c64, bnd) <= 1.0
        assert freivalds(out, ta, tb, n, n, n, 1.5, A, lda, B, ldb, -0.25, C, ldc, seed=8) <= 1.0


_LINPACK_C = {}


@pytest.mark.parametrize("nb", [128, 256])
def test_linpack_trailing_update_16384(h, nb):
    """The Linpack-shaped update at m = n = 16384 (seed 2, entries normal(0,1)
    times 2^e per stored row, e in [-20, 20]), against the CPU oracle on
    sampled 256 x 256 blocks and by the Freivalds identity over the whole
    result."""
    import torch
    m = n = 16384
    if m not in _LINPACK_C:
        _LINPACK_C[m] = synth.normal_rowscaled_matrix(2, 4, m, n, m)
    C = _LINPACK_C[m]
    A = synth.normal_rowscaled_matrix(2, 0, m, nb, m)
    B = synth.normal_rowscaled_matrix(2, 2, nb, n, nb)
    dA, dB, dC = dev(A), dev(B), dev(C)
    h.set_path(0)  # AUTO: k = nb >= 128 runs the split path
    h.sgemm("N", "N", m, n, nb, -1.0, dA, m, dB, nb, 1.0, dC, m)
    torch.cuda.synchronize()
    assert h.last_path() == SPLIT and h.get_device_status() == 0
    out = dC.cpu().numpy()
    del dA, dB, dC
    got = synth.logical(out, m, n, m)
    for rows, cols in sample_blocks(m, n, 256, seed=9, count=3):
        c64, bnd = O.gemm_f64("N", "N", m, n, nb, -1.0, A, m, B, nb, 1.0, C, m, rows=rows, cols=cols)
        assert O.error_ratio(got[rows[0]:rows[1], cols[0]:cols[1]], c64, bnd) <= 1.0
    assert freivalds(out, "N", "N", m, n, nb, -1.0, A, m, B, nb, 1.0, C, m, seed=10) <= 1.0
