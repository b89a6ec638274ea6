"""Helpers for the GPU parity tests: run the C-ABI sgemm on seeded inputs and
compare with the CPU oracle (FP64) under the componentwise bound."""

from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

SIMT = 1
SPLIT = 2


def dev(x: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_sgemm(h, path, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, null_ab=False):
    """Copy inputs to the device, run gbgemm_sgemm on `path`, return C as numpy."""
    import torch
    h.set_path(path)
    dA = None if null_ab else dev(A)
    dB = None if null_ab else dev(B)
    dC = dev(C)
    h.sgemm(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc)
    torch.cuda.synchronize()
    assert h.get_device_status() == 0
    return dC.cpu().numpy()


def check_full(h, path, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, max_ratio=1.0, nthreads=0):
    """Run and compare every entry with the oracle; returns the max error ratio."""
    out = run_sgemm(h, path, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
    assert synth.padding_is_sentinel(out, m, n, ldc), "write outside the logical C"
    if m == 0 or n == 0:
        assert np.array_equal(out.view(np.uint32), C.view(np.uint32))
        return 0.0
    c64, bnd = O.gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=nthreads)
    got = synth.logical(out, m, n, ldc)
    r = O.error_ratio(got, c64, bnd)
    assert r <= max_ratio, f"path={path} {ta}{tb} m={m} n={n} k={k}: ratio {r}"
    return r


def sample_blocks(m, n, bs, seed, count=4):
    """Corner and diagonal blocks plus `count` seeded random ones (row range, col range)."""
    bm, bn = min(bs, m), min(bs, n)
    starts = [(0, 0), (m - bm, n - bn), (0, n - bn), (m - bm, 0), ((m - bm) // 2, (n - bn) // 2)]
    u = synth.draws(seed, 50, 2 * count)
    for t in range(count):
        starts.append((int(u[2 * t] % np.uint64(m - bm + 1)), int(u[2 * t + 1] % np.uint64(n - bn + 1))))
    return [((i, i + bm), (j, j + bn)) for i, j in starts]


def check_sampled(out, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, bs=256, seed=0, count=3):
    """Oracle on sampled blocks of a large output; returns the max error ratio."""
    worst = 0.0
    got = synth.logical(out, m, n, ldc)
    for rows, cols in sample_blocks(m, n, bs, seed, count):
        c64, bnd = O.gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, rows=rows, cols=cols)
        r = O.error_ratio(got[rows[0]:rows[1], cols[0]:cols[1]], c64, bnd)
        worst = max(worst, r)
    return worst


def freivalds(out, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, seed=0):
    ar, ac = synth.op_shape(ta, m, k)
    br, bc = synth.op_shape(tb, k, n)
    Am = synth.logical(A, ar, ac, lda)
    Bm = synth.logical(B, br, bc, ldb)
    opA = Am if ta in "Nn" else Am.T
    opB = Bm if tb in "Nn" else Bm.T
    x = np.where((synth.draws(seed, 60, n) >> np.uint64(63)) == 1, 1.0, -1.0)
    return O.freivalds_ratio(opA, opB, synth.logical(C, m, n, ldc), synth.logical(out, m, n, ldc), alpha, beta, x)
