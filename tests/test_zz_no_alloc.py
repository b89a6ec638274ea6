"""The allocation-free split sgemm (gbgemm_sgemm_split_noalloc).

It serves callers that cannot call cudaMalloc when they multiply (inside
another component's stream capture, inside allocator callbacks, in
latency-bound loops, or with device memory reserved by another framework):
its scratch is a fixed array in the library's device memory instead of a
handle's workspace.  This file is named so that pytest collects it last.

Checks, through the C ABI, on calls in a row (each reuses the scratch the
one before left behind):
  * the result of the allocation-free call is within the acceptance bound
    |C - C64| <= 2 k 2^-24 (|alpha||A||B| + |beta||C|) of the FP64 oracle,
    element by element, as is that of gbgemm_sgemm on the split path;
  * the two results agree with each other within the same bound;
  * the cases cover the three-part split (k < 512), the two-part split
    (k >= 512) and operands whose rows span 2^-60 .. 2^60 (the re-pack of
    badly scaled K-vectors writes into the scratch panels too);
a problem needing more scratch than the fixed maximum is refused with
GBGEMM_ERR_SCRATCH_LIMIT before anything runs.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

pytestmark = pytest.mark.gpu


def _scaled(seed, ta, tb, m, n, k, pad):
    """Uniform operands whose K-vectors are scaled by 2^e, e in [-60, 60]:
    rows of op(A) and columns of op(B)."""
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", seed, ta, tb, m, n, k, pad=pad)
    ea = synth.int_range(synth.draws(seed, 80, m), -60, 60)
    eb = synth.int_range(synth.draws(seed, 81, n), -60, 60)
    ar, ac = synth.op_shape(ta, m, k)
    br, bc = synth.op_shape(tb, k, n)
    Al = synth.logical(A, ar, ac, lda).astype(np.float64)
    Bl = synth.logical(B, br, bc, ldb).astype(np.float64)
    Al = Al * (np.ldexp(1.0, ea)[:, None] if ta in "Nn" else np.ldexp(1.0, ea)[None, :])
    Bl = Bl * (np.ldexp(1.0, eb)[None, :] if tb in "Nn" else np.ldexp(1.0, eb)[:, None])
    A2, B2 = A.copy(), B.copy()
    synth.logical(A2, ar, ac, lda)[...] = Al.astype(np.float32)
    synth.logical(B2, br, bc, ldb)[...] = Bl.astype(np.float32)
    return A2, lda, B2, ldb, C, ldc


def _run_both(L, h, stream, ta, tb, m, n, k, alpha, beta, seed, scaled=False):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    if scaled:
        A, lda, B, ldb, C, ldc = _scaled(seed, ta, tb, m, n, k, pad=3)
    else:
        A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", seed, ta, tb, m, n, k, pad=3)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    c_new = torch.from_numpy(C).cuda()
    c_old = torch.from_numpy(C).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = L.gbgemm_sgemm_split_noalloc(stream, ta.encode(), tb.encode(), m, n, k, alpha, dA.data_ptr(), lda,
                                      dB.data_ptr(), ldb, beta, c_new.data_ptr(), ldc, status.data_ptr())
    assert rc == gbgemm.OK, gbgemm.status_string(rc)
    h.set_path(gbgemm.PATH_SPLIT_BF16)
    h.sgemm(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, c_old, ldc)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert h.get_device_status() == 0
    new = c_new.cpu().numpy()
    old = c_old.cpu().numpy()
    assert synth.padding_is_sentinel(new, m, n, ldc)
    c64, bound = O.gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
    got_new = synth.logical(new, m, n, ldc)
    got_old = synth.logical(old, m, n, ldc)
    assert O.error_ratio(got_new, c64, bound) <= 1.0
    assert O.error_ratio(got_old, c64, bound) <= 1.0
    diff = np.abs(got_new.astype(np.float64) - got_old)
    assert np.all(diff <= bound)


def test_noalloc_matches_oracle_and_existing_entry_point_in_a_row():
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    L = gbgemm.lib()
    h = gbgemm.Handle(0)
    stream = torch.cuda.current_stream()
    h.set_stream(stream)
    # three-part split (k < 512), then a larger two-part one that reuses what
    # the first left in the scratch array, then badly scaled operands (re-pack)
    # on both splits
    _run_both(L, h, stream.cuda_stream, "N", "T", 300, 520, 384, 1.5, -0.25, 41)
    _run_both(L, h, stream.cuda_stream, "T", "N", 1000, 777, 555, -1.0, 1.0, 42)
    _run_both(L, h, stream.cuda_stream, "N", "N", 257, 300, 200, 1.0, 0.5, 43, scaled=True)
    _run_both(L, h, stream.cuda_stream, "T", "T", 390, 260, 640, 2.0, 0.0, 44, scaled=True)
    h.close()


def test_noalloc_refuses_problems_beyond_the_scratch_limit():
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    L = gbgemm.lib()
    n = 4096  # needs 2 x 128 MiB of panels: beyond the 64 MiB array
    assert gbgemm.split_workspace_bytes(n, n, n) + 256 > gbgemm.NOALLOC_SCRATCH_BYTES
    A = torch.zeros(n * n, device="cuda")
    B = torch.zeros(n * n, device="cuda")
    C = torch.full((n * n,), 7.0, device="cuda")
    rc = L.gbgemm_sgemm_split_noalloc(torch.cuda.current_stream().cuda_stream, b"N", b"N", n, n, n, 1.0,
                                      A.data_ptr(), n, B.data_ptr(), n, 0.0, C.data_ptr(), n, None)
    torch.cuda.synchronize()
    assert rc == gbgemm.ERR_SCRATCH_LIMIT
    assert bool(torch.all(C == 7.0))
