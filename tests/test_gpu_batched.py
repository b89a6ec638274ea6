"""GPU parity of the strided-batched sgemm: every problem of the batch against
the FP64 oracle under the acceptance bound, both paths, every transpose,
shared operands (stride 0), padding untouched, degenerate batches."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

from gpu_util import SIMT, SPLIT, dev

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


def batch_data(seed, ta, tb, m, n, k, batch, pad=3, share_a=False, share_b=False, gap=7):
    """Column-major operands of `batch` problems laid end to end (stride = one
    problem's storage + gap), the gaps filled with the padding sentinel."""
    ar, ac = synth.op_shape(ta, m, k)
    br, bc = synth.op_shape(tb, k, n)
    lda, ldb, ldc = ar + pad, br + pad, m + pad
    sa = 0 if share_a else lda * ac + gap
    sb = 0 if share_b else ldb * bc + gap
    sc = ldc * n + gap
    def stack(rows, cols, ld, stride, count, s0):
        total = stride * (count - 1) + ld * cols if count > 0 else 0
        buf = np.full(max(total, ld * cols), np.float32(0.0)).view(np.uint32)
        buf[:] = 0x7FC0FFEE
        buf = buf.view(np.float32)
        mats = []
        for z in range(count if stride > 0 else 1):
            X = synth.uniform_matrix(seed, s0 + 2 * z, rows, cols, ld)
            buf[z * stride: z * stride + ld * cols] = X
            mats.append(X)
        return buf, mats
    A, As = stack(ar, ac, lda, sa, batch, 0)
    B, Bs = stack(br, bc, ldb, sb, batch, 1000)
    C, Cs = stack(m, n, ldc, sc, batch, 2000)
    return A, lda, sa, As, B, ldb, sb, Bs, C, ldc, sc, Cs


def check_batch(h, path, ta, tb, m, n, k, alpha, beta, batch, **kw):
    import torch
    A, lda, sa, As, B, ldb, sb, Bs, C, ldc, sc, Cs = batch_data(11, ta, tb, m, n, k, batch, **kw)
    dA, dB, dC = dev(A), dev(B), dev(C)
    h.set_path(path)
    h.sgemm_strided_batched(ta, tb, m, n, k, alpha, dA, lda, sa, dB, ldb, sb, beta, dC, ldc, sc, batch)
    torch.cuda.synchronize()
    assert h.get_device_status() == 0
    out = dC.cpu().numpy()
    worst = 0.0
    for z in range(batch):
        Az = As[z if sa else 0]
        Bz = Bs[z if sb else 0]
        Cz = Cs[z]
        oz = out[z * sc: z * sc + ldc * n]
        assert synth.padding_is_sentinel(oz, m, n, ldc)
        c64, bnd = O.gemm_f64(ta, tb, m, n, k, alpha, Az, lda, Bz, ldb, beta, Cz, ldc)
        r = O.error_ratio(synth.logical(oz, m, n, ldc), c64, bnd)
        assert r <= 1.0, (path, ta, tb, m, n, k, z, r)
        worst = max(worst, r)
    # the gaps between results are untouched
    for z in range(batch - 1):
        gap = out[z * sc + ldc * n: (z + 1) * sc].view(np.uint32)
        assert np.all(gap == 0x7FC0FFEE)
    return worst


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("path", [SIMT, SPLIT])
def test_batched_every_transpose(h, path, ta, tb):
    check_batch(h, path, ta, tb, 150, 130, 300, 1.5, -0.25, 5)


@pytest.mark.parametrize("path", [SIMT, SPLIT])
def test_batched_long_k_and_shared_operands(h, path):
    # k >= 512: two-part split; A shared by every problem
    check_batch(h, path, "N", "N", 200, 70, 700, 1.0, 0.0, 4, share_a=True)
    # B shared, three-part split, odd sizes
    check_batch(h, path, "T", "N", 129, 257, 160, -1.0, 1.0, 3, share_b=True)


def test_batched_auto_path_and_degenerate(h):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    # AUTO: k < 128 runs SIMT, k >= 128 the split path
    check_batch(h, gbgemm.PATH_AUTO, "N", "T", 90, 60, 40, 1.0, 0.5, 6)
    assert h.last_path() == SIMT
    check_batch(h, gbgemm.PATH_AUTO, "N", "N", 90, 60, 256, 1.0, 0.5, 6)
    assert h.last_path() == SPLIT
    # alpha = 0: C := beta C for every problem, A and B not read
    A, lda, sa, As, B, ldb, sb, Bs, C, ldc, sc, Cs = batch_data(12, "N", "N", 40, 30, 20, 3)
    dC = dev(C)
    h.sgemm_strided_batched("N", "N", 40, 30, 20, 0.0, None, lda, sa, None, ldb, sb, 2.0, dC, ldc, sc, 3)
    torch.cuda.synchronize()
    out = dC.cpu().numpy()
    for z in range(3):
        oz = synth.logical(out[z * sc: z * sc + ldc * 30], 40, 30, ldc)
        assert np.array_equal(oz, (2.0 * synth.logical(Cs[z], 40, 30, ldc)).astype(np.float32))
    # batch 0 and empty problems return without touching anything
    assert h.sgemm_strided_batched("N", "N", 40, 30, 20, 1.0, None, lda, sa, None, ldb, sb, 0.0, None, ldc, sc, 0) == 0
    assert h.sgemm_strided_batched("N", "N", 0, 30, 20, 1.0, None, 1, 0, None, 20, 0, 0.0, None, 1, 0, 5) == 0


def test_batched_matches_single_calls(h):
    """A batch and the same problems called one by one agree bit for bit (the
    same kernels and configuration; k < 512, where single calls are not cut
    into k slices)."""
    import torch
    m, n, k, batch = 256, 256, 384, 3
    A, lda, sa, As, B, ldb, sb, Bs, C, ldc, sc, Cs = batch_data(13, "N", "N", m, n, k, batch)
    dA, dB, dC, dC1 = dev(A), dev(B), dev(C), dev(C)
    h.set_path(SPLIT)
    h.sgemm_strided_batched("N", "N", m, n, k, 1.0, dA, lda, sa, dB, ldb, sb, 0.5, dC, ldc, sc, batch)
    for z in range(batch):
        h.sgemm("N", "N", m, n, k, 1.0, dA[z * sa:], lda, dB[z * sb:], ldb, 0.5, dC1[z * sc:], ldc)
    torch.cuda.synchronize()
    assert np.array_equal(dC.cpu().numpy().view(np.uint32), dC1.cpu().numpy().view(np.uint32))
