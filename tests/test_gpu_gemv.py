"""GPU parity of sgemv: y := alpha op(A) x + beta y against the FP64 oracle
(gemv is the gemm of op(A) with one column), under the acceptance bound with
k the summed length; both transposes, positive, negative and strided
increments, sliced and unsliced launches, degenerate cases, determinism."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

from gpu_util import dev

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


def strided(v, inc):
    """BLAS storage of vector v with increment inc (sentinels between)."""
    n = len(v)
    buf = np.full(max(1, 1 + (n - 1) * abs(inc)), np.float32(0.0)).view(np.uint32)
    buf[:] = 0x7FC0FFEE
    buf = buf.view(np.float32)
    for e in range(n):
        buf[e * inc if inc > 0 else (n - 1 - e) * (-inc)] = v[e]
    return buf


def gather(buf, n, inc):
    return np.array([buf[e * inc if inc > 0 else (n - 1 - e) * (-inc)] for e in range(n)], dtype=np.float32)


def check_gemv(h, trans, m, n, alpha, beta, incx=1, incy=1, pad=3, seed=21):
    import torch
    lda = m + pad
    A = synth.uniform_matrix(seed, 0, m, n, lda)
    lx, ly = (m, n) if trans == "T" else (n, m)
    xv = synth.uniform_pm1(synth.draws(seed, 2, max(lx, 1)))[:lx].astype(np.float32)
    yv = synth.uniform_pm1(synth.draws(seed, 3, max(ly, 1)))[:ly].astype(np.float32)
    xb, yb = strided(xv, incx), strided(yv, incy)
    dA, dx, dy = dev(A), dev(xb), dev(yb)
    h.sgemv(trans, m, n, alpha, dA, lda, dx, incx, beta, dy, incy)
    torch.cuda.synchronize()
    out = dy.cpu().numpy()
    # entries of the y storage that are not vector elements are untouched
    mask = np.ones(len(yb), bool)
    for e in range(ly):
        mask[e * incy if incy > 0 else (ly - 1 - e) * (-incy)] = False
    assert np.array_equal(out.view(np.uint32)[mask], yb.view(np.uint32)[mask])
    got = gather(out, ly, incy)
    if ly == 0:
        return 0.0, out
    # oracle: op(A) (ly x lx) times x (lx x 1), plus beta y
    c64, bnd = O.gemm_f64(trans, "N", ly, 1, lx, alpha, A, lda, xv.copy(), max(lx, 1), beta, yv.copy(), max(ly, 1))
    r = O.error_ratio(got.reshape(ly, 1), c64, bnd)
    assert r <= 1.0, (trans, m, n, incx, incy, r)
    return r, out


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("m,n", [(1, 1), (300, 7), (7, 300), (1000, 2000), (5000, 40), (40, 5000), (257, 1031)])
def test_gemv_against_oracle(h, trans, m, n):
    check_gemv(h, trans, m, n, 1.5, -0.25)


@pytest.mark.parametrize("incx,incy", [(2, 3), (-1, 1), (1, -2), (-3, -1)])
def test_gemv_increments(h, incx, incy):
    check_gemv(h, "N", 600, 900, 0.75, 0.5, incx=incx, incy=incy)
    check_gemv(h, "T", 600, 900, 0.75, 0.5, incx=incx, incy=incy)


def test_gemv_alpha_beta_and_empty(h):
    import torch
    # alpha = 0: y := beta y, A and x not read
    yv = synth.uniform_pm1(synth.draws(22, 3, 50)).astype(np.float32)
    dy = dev(yv)
    h.sgemv("N", 50, 20, 0.0, None, 50, None, 1, 2.0, dy, 1)
    torch.cuda.synchronize()
    assert np.array_equal(dy.cpu().numpy(), (2.0 * yv).astype(np.float32))
    # beta = 0: y is not read (NaN stays out)
    r, _ = check_gemv(h, "T", 300, 200, 1.0, 0.0)
    assert r <= 1.0
    dy = dev(np.full(50, np.nan, np.float32))
    dA, dx = dev(synth.uniform_matrix(23, 0, 50, 20, 50)), dev(np.ones(20, np.float32))
    h.sgemv("N", 50, 20, 1.0, dA, 50, dx, 1, 0.0, dy, 1)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(dy.cpu().numpy()))
    # empty: nothing launched, nothing touched
    assert h.sgemv("N", 0, 20, 1.0, None, 1, None, 1, 0.0, None, 1) == 0
    assert h.sgemv("T", 0, 20, 1.0, None, 1, None, 1, 0.5, dy, 1) == 0  # x empty: y := 0.5 y
    torch.cuda.synchronize()


def test_gemv_deterministic(h):
    _, a = check_gemv(h, "N", 300, 60000, 1.0, 0.0, seed=24)   # sliced columns
    _, b = check_gemv(h, "N", 300, 60000, 1.0, 0.0, seed=24)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    _, a = check_gemv(h, "T", 60000, 30, 1.0, 0.0, seed=25)    # sliced rows
    _, b = check_gemv(h, "T", 60000, 30, 1.0, 0.0, seed=25)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
