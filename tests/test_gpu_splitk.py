"""Split-K on the split path: single calls whose output has too few tiles for
the SMs are cut into k slices whose raw accumulators a reduction sums in slice
order.  Checked against the FP64 oracle under the acceptance bound, with
badly scaled rows, for run-to-run determinism, and for the launches made."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

from gpu_util import SPLIT, check_full, dev

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


def launches(h, fn):
    import torch
    h.profile_begin()
    fn()
    torch.cuda.synchronize()
    return h.profile_end()[2]


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_splitk_against_oracle(h, ta, tb):
    m, n, k = 200, 150, 8192  # 6 tiles of 128 x 64 for 152 SMs: sliced
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 91, ta, tb, m, n, k, pad=3)
    assert check_full(h, SPLIT, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc, nthreads=4) <= 1.0


def test_splitk_badly_scaled_rows(h):
    """Row scales 2^+-60 on op(A) and op(B): the reduction applies 2^(e_i + f_j)."""
    m, n, k = 150, 130, 4096
    A = synth.normal_rowscaled_matrix(92, 0, m, k, m, elo=-60, ehi=60)
    Bt = synth.normal_rowscaled_matrix(92, 2, n, k, n, elo=-60, ehi=60)  # op(B) columns scaled: B stored T
    C = synth.uniform_matrix(92, 4, m, n, m)
    assert check_full(h, SPLIT, "N", "T", m, n, k, 1.0, A, m, Bt, n, 0.5, C, m, nthreads=4) <= 1.0


def test_splitk_deterministic_and_launches(h):
    import torch
    m, n, k = 256, 256, 16384
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 93, "N", "N", m, n, k, pad=0)
    dA, dB = dev(A), dev(B)
    outs = []
    h.set_path(SPLIT)
    for _ in range(2):
        dC = dev(C)
        n_launch = launches(h, lambda: h.sgemm("N", "N", m, n, k, 1.0, dA, lda, dB, ldb, 0.5, dC, ldc))
        # the packing of both operands, the GEMM and the split-K reduction
        assert n_launch == 3
        outs.append(dC.cpu().numpy())
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))
    c64, bnd = O.gemm_f64("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc, nthreads=4)
    assert O.error_ratio(synth.logical(outs[0], m, n, ldc), c64, bnd) <= 1.0
    # enough tiles for the SMs, or k below 512: no slicing
    m2, n2, k2 = 2048, 2048, 1024
    A2, lda2, B2, ldb2, C2, ldc2 = synth.gemm_problem("uniform", 94, "N", "N", m2, n2, k2, pad=0)
    dA2, dB2, dC2 = dev(A2), dev(B2), dev(C2)
    assert launches(h, lambda: h.sgemm("N", "N", m2, n2, k2, 1.0, dA2, lda2, dB2, ldb2, 0.0, dC2, ldc2)) == 2
    A3, lda3, B3, ldb3, C3, ldc3 = synth.gemm_problem("uniform", 95, "N", "N", 100, 100, 300, pad=0)
    dA3, dB3, dC3 = dev(A3), dev(B3), dev(C3)
    assert launches(h, lambda: h.sgemm("N", "N", 100, 100, 300, 1.0, dA3, lda3, dB3, ldb3, 0.0, dC3, ldc3)) == 2
