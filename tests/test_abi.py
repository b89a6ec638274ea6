"""The C-ABI library: builds, loads, exports every declared symbol, and
rejects bad arguments in BLAS order without touching a GPU."""

import ctypes
import os
import re

import pytest

from paper_1608_05265_gb300 import build, gbgemm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return gbgemm.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "gbgemm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gbgemm_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
    assert sorted(gbgemm.EXPORTS) == names


def test_argument_errors_in_blas_order(L):
    a = ctypes.c_void_p(16)  # never dereferenced: argument checks run first
    sg = L.gbgemm_sgemm
    assert sg(None, b"X", b"N", 1, 1, 1, 1.0, a, 1, a, 1, 0.0, a, 1) == -1
    assert sg(None, b"N", b"q", 1, 1, 1, 1.0, a, 1, a, 1, 0.0, a, 1) == -2
    assert sg(None, b"N", b"N", -1, 1, 1, 1.0, a, 1, a, 1, 0.0, a, 1) == -3
    assert sg(None, b"N", b"N", 1, -1, 1, 1.0, a, 1, a, 1, 0.0, a, 1) == -4
    assert sg(None, b"N", b"N", 1, 1, -1, 1.0, a, 1, a, 1, 0.0, a, 1) == -5
    assert sg(None, b"N", b"N", 5, 1, 3, 1.0, a, 4, a, 3, 0.0, a, 5) == -8
    assert sg(None, b"T", b"N", 5, 1, 3, 1.0, a, 2, a, 3, 0.0, a, 5) == -8
    assert sg(None, b"N", b"N", 5, 2, 3, 1.0, a, 5, a, 2, 0.0, a, 5) == -10
    assert sg(None, b"N", b"T", 5, 2, 3, 1.0, a, 5, a, 1, 0.0, a, 5) == -10
    assert sg(None, b"N", b"N", 5, 2, 3, 1.0, a, 5, a, 3, 0.0, a, 4) == -13
    assert sg(None, b"N", b"N", 5, 2, 3, 1.0, None, 5, a, 3, 0.0, a, 5) == -7
    assert sg(None, b"N", b"N", 5, 2, 3, 1.0, a, 5, None, 3, 0.0, a, 5) == -9
    assert sg(None, b"N", b"N", 5, 2, 3, 1.0, a, 5, a, 3, 0.0, None, 5) == -12
    # ld of 0 is invalid even for empty matrices (BLAS requires ld >= 1)
    assert sg(None, b"N", b"N", 0, 0, 0, 1.0, a, 0, a, 1, 0.0, a, 1) == -8
    # alpha == 0: A and B may be null; then the handle is checked
    assert sg(None, b"N", b"N", 5, 2, 3, 0.0, None, 5, None, 3, 2.0, a, 5) == gbgemm.ERR_NOT_INITIALIZED
    # every letter of the transpose alphabet is accepted
    for ta in b"NnTtCc":
        assert sg(None, bytes([ta]), b"n", 1, 1, 1, 1.0, a, 1, a, 1, 0.0, a, 1) == gbgemm.ERR_NOT_INITIALIZED


def test_batched_argument_errors_in_order(L):
    a = ctypes.c_void_p(16)  # never dereferenced: argument checks run first
    sb = L.gbgemm_sgemm_strided_batched
    def call(ta=b"N", tb=b"N", m=5, n=2, k=3, alpha=1.0, A=a, lda=5, sa=15, B=a, ldb=3, sbb=6, beta=0.0, C=a,
             ldc=5, sc=10, batch=4):
        return sb(None, ta, tb, m, n, k, alpha, A, lda, sa, B, ldb, sbb, beta, C, ldc, sc, batch)
    assert call(ta=b"X") == -1
    assert call(tb=b"q") == -2
    assert call(m=-1) == -3
    assert call(n=-1) == -4
    assert call(k=-1) == -5
    assert call(lda=4) == -8
    assert call(sa=-1) == -9
    assert call(ldb=2) == -11
    assert call(sbb=-3) == -12
    assert call(ldc=4) == -15
    assert call(sc=-1) == -16
    assert call(sc=9) == -16          # C_1 would overlap C_0 (needs ldc (n - 1) + m = 10)
    assert call(batch=-1) == -17
    assert call(batch=65536) == -17
    assert call(A=None) == -7
    assert call(B=None) == -10
    assert call(C=None) == -14
    # shared operands (stride 0) and one problem (any stride_c) are fine
    assert call(sa=0, sbb=0) == gbgemm.ERR_NOT_INITIALIZED
    assert call(sc=0, batch=1) == gbgemm.ERR_NOT_INITIALIZED
    assert call(batch=0) == gbgemm.ERR_NOT_INITIALIZED


def test_gemv_argument_errors_in_order(L):
    a = ctypes.c_void_p(16)  # never dereferenced: argument checks run first
    gv = L.gbgemm_sgemv
    def call(t=b"N", m=5, n=3, alpha=1.0, A=a, lda=5, x=a, incx=1, beta=0.0, y=a, incy=1):
        return gv(None, t, m, n, alpha, A, lda, x, incx, beta, y, incy)
    assert call(t=b"Q") == -1
    assert call(m=-1) == -2
    assert call(n=-1) == -3
    assert call(lda=4) == -6
    assert call(incx=0) == -8
    assert call(incy=0) == -11
    assert call(A=None) == -5
    assert call(x=None) == -7
    assert call(y=None) == -10
    assert call(alpha=0.0, A=None, x=None, beta=2.0) == gbgemm.ERR_NOT_INITIALIZED
    assert call(incx=-2, incy=-1) == gbgemm.ERR_NOT_INITIALIZED
    for t in b"NnTtCc":
        assert call(t=bytes([t])) == gbgemm.ERR_NOT_INITIALIZED


def test_getrf_getrs_argument_errors_in_order(L):
    a = ctypes.c_void_p(16)  # never dereferenced: argument checks run first
    def getrf(n=5, A=a, lda=5, ipiv=a, info=a, nb=0):
        return L.gbgemm_sgetrf(None, n, A, lda, ipiv, info, nb)
    assert getrf(n=-1) == -1
    assert getrf(n=2**31) == -1
    assert getrf(A=None) == -2
    assert getrf(lda=4) == -3
    assert getrf(ipiv=None) == -4
    assert getrf(info=None) == -5
    assert getrf(nb=-1) == -6
    assert getrf(nb=129) == -6
    assert getrf(n=0, A=None, lda=1, ipiv=None) == gbgemm.ERR_NOT_INITIALIZED
    assert getrf(nb=128) == gbgemm.ERR_NOT_INITIALIZED
    def getrs(n=5, nrhs=2, LU=a, lda=5, ipiv=a, B=a, ldb=5):
        return L.gbgemm_sgetrs(None, n, nrhs, LU, lda, ipiv, B, ldb)
    assert getrs(n=-1) == -1
    assert getrs(nrhs=-1) == -2
    assert getrs(LU=None) == -3
    assert getrs(lda=4) == -4
    assert getrs(ipiv=None) == -5
    assert getrs(B=None) == -6
    assert getrs(ldb=4) == -7
    assert getrs(nrhs=0, B=None) == gbgemm.ERR_NOT_INITIALIZED
    assert getrs() == gbgemm.ERR_NOT_INITIALIZED


def test_null_handle_and_status_strings(L):
    assert L.gbgemm_destroy(None) == gbgemm.ERR_NOT_INITIALIZED
    assert L.gbgemm_set_path(None, 0) == gbgemm.ERR_NOT_INITIALIZED
    assert L.gbgemm_create(None, 0) == gbgemm.ERR_INVALID_VALUE
    for s in (0, -3, -100, -101, -102, -103, -104, -105, -106, 7):
        assert isinstance(gbgemm.status_string(s), str) and gbgemm.status_string(s)
    assert gbgemm.status_string(-104) == "GBGEMM_ERR_DEVICE_TIMEOUT"


def test_panel_and_workspace_sizes(L):
    # 16 KiB blocks, rows rounded up to a multiple of 256, k to a multiple of 32
    assert gbgemm.panel_bytes(1, 1) == 2 * 16384
    assert gbgemm.panel_bytes(256, 32) == 2 * 16384
    assert gbgemm.panel_bytes(257, 33) == 4 * 2 * 16384
    assert gbgemm.panel_bytes(8192, 8192) == 64 * 256 * 16384
    assert gbgemm.panel_bytes(0, 5) == 0
    ws = gbgemm.split_workspace_bytes(8192, 8192, 8192)
    # control words (256 B), 64 + 64 band counters (512 B), row maxima, panels
    assert ws == 256 + 512 + 2 * 8192 * 4 + 2 * 64 * 256 * 16384
    # three parts below k = 512: a compact lo3 panel per operand as well
    assert gbgemm.split_workspace_bytes(300, 200, 100) == 256 + 256 + 2048 + 2 * (4 + 2) * 4 * 16384


def test_no_cpu_fallback_without_gpu(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert L.gbgemm_create(ctypes.byref(h), 0) == gbgemm.ERR_CUDA


def test_schedule_table(L):
    # 3 SIMT schedules, then split schedules 3 + 12 b + 4 r + q (BN 64 << b, R in 1/4/16, k-slicing level q)
    seen = set()
    for s in range(gbgemm.NUM_SCHEDULES):
        d = gbgemm.schedule_info(s)
        if s < 3:
            assert d["path"] == gbgemm.PATH_SIMT and (d["tile_m"], d["tile_n"]) == [(128, 128), (64, 64), (128, 64)][s]
            continue
        b, r, q = (s - 3) // 12, ((s - 3) // 4) % 3, (s - 3) % 4
        assert d == {"path": gbgemm.PATH_SPLIT_BF16, "tile_m": 128, "tile_n": 64 << b, "raster": (1, 4, 16)[r],
                     "level": q}
        seen.add((d["tile_n"], d["raster"], d["level"]))
    assert len(seen) == 36 and gbgemm.NUM_SCHEDULES == 39
    for bad in (-1, 39, 1000):
        with pytest.raises(gbgemm.GbgemmError):
            gbgemm.schedule_info(bad)
    a = ctypes.c_void_p(16)
    assert L.gbgemm_set_schedule(None, 3) == gbgemm.ERR_NOT_INITIALIZED
    assert L.gbgemm_predictor_select(None, 1) == gbgemm.ERR_NOT_INITIALIZED
