"""Python access to the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg import this module.  The product library never does.

The arithmetic lives in ``ref_gemm.c`` (plain C loops, see its header for the
definitions and the passages they follow).  This module builds it with gcc
and marshals numpy arrays; it adds a few derived checks written in numpy
float64 (the Freivalds identity used for full-size outputs).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ref_gemm.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ref_gemm.c into oracle/_build/liboracle.so (OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, f32, vp = ctypes.c_int64, ctypes.c_float, ctypes.c_void_p
            L.oracle_gemm_f64.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64, f32, vp, i64, vp, i64,
                                          f32, vp, i64, i64, i64, i64, i64, vp, i64, vp, ctypes.c_int]
            L.oracle_gemm_f64.restype = ctypes.c_int
            L.oracle_gemm_f32.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64, f32, vp, i64, vp, i64,
                                          f32, vp, i64, i64, i64, i64, i64, vp, i64, ctypes.c_int]
            L.oracle_gemm_f32.restype = ctypes.c_int
            L.oracle_bf16_rne.argtypes = [f32]
            L.oracle_bf16_rne.restype = ctypes.c_uint16
            L.oracle_scale_exponent.argtypes = [f32]
            L.oracle_scale_exponent.restype = ctypes.c_int
            L.oracle_split_rows.argtypes = [i64, i64, vp, i64, i64, vp, vp, vp]
            L.oracle_split_rows.restype = None
            L.oracle_split_exhaustive.argtypes = [ctypes.c_uint64, ctypes.c_uint64, vp, ctypes.c_int]
            L.oracle_split3_exhaustive.argtypes = [ctypes.c_uint64, ctypes.c_uint64, vp, ctypes.c_int]
            L.oracle_split3_exhaustive.restype = None
            L.oracle_split_rows3.argtypes = [i64, i64, vp, i64, i64, vp, vp, vp, vp]
            L.oracle_split_rows3.restype = None
            L.oracle_split_third.argtypes = [f32]
            L.oracle_split_third.restype = ctypes.c_uint16
            L.oracle_split_exhaustive.restype = None
            L.oracle_max_threads.restype = ctypes.c_int
            L.oracle_trans_code.argtypes = [ctypes.c_char]
            L.oracle_trans_code.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def gemm_f64(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
             rows=None, cols=None, nthreads=0, want_bound=True):
    """FP64 result (and acceptance bound) of the block rows x cols of C_out.

    ``rows`` / ``cols`` are (start, stop) ranges, default the whole matrix.
    Returns (out, bound) as float64 arrays indexed [i - i0, j - j0].
    """
    i0, i1 = rows if rows is not None else (0, m)
    j0, j1 = cols if cols is not None else (0, n)
    bm, bn = i1 - i0, j1 - j0
    out = np.zeros((max(bn, 1), max(bm, 1)), dtype=np.float64)  # column-major block
    bnd = np.zeros_like(out) if want_bound else None
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    C = np.ascontiguousarray(C, dtype=np.float32)
    rc = lib().oracle_gemm_f64(transa.encode(), transb.encode(), m, n, k, float(alpha), _ptr(A), lda, _ptr(B), ldb,
                               float(beta), _ptr(C), ldc, i0, i1, j0, j1, _ptr(out), max(bm, 1),
                               _ptr(bnd) if bnd is not None else None, int(nthreads))
    if rc != 0:
        raise ValueError("bad transpose flag")
    out = out.T[:bm, :bn]
    return (out, bnd.T[:bm, :bn] if bnd is not None else None)


def gemm_f32(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, rows=None, cols=None, nthreads=0):
    i0, i1 = rows if rows is not None else (0, m)
    j0, j1 = cols if cols is not None else (0, n)
    bm, bn = i1 - i0, j1 - j0
    out = np.zeros((max(bn, 1), max(bm, 1)), dtype=np.float32)
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    C = np.ascontiguousarray(C, dtype=np.float32)
    rc = lib().oracle_gemm_f32(transa.encode(), transb.encode(), m, n, k, float(alpha), _ptr(A), lda, _ptr(B), ldb,
                               float(beta), _ptr(C), ldc, i0, i1, j0, j1, _ptr(out), max(bm, 1), int(nthreads))
    if rc != 0:
        raise ValueError("bad transpose flag")
    return out.T[:bm, :bn]


def bf16_rne(x: float) -> int:
    return int(lib().oracle_bf16_rne(float(x)))


def scale_exponent(amax: float) -> int:
    return int(lib().oracle_scale_exponent(float(amax)))


def split_rows(X: np.ndarray, rows: int, k: int, sr: int, sp: int):
    """Split ``rows`` K-vectors (element (r,p) = X[r*sr + p*sp]) into (e, hi, lo).

    hi and lo are uint16 bfloat16 patterns, shape (rows, k).
    """
    X = np.ascontiguousarray(X, dtype=np.float32)
    e = np.zeros(max(rows, 1), dtype=np.int32)
    hi = np.zeros((max(rows, 1), max(k, 1)), dtype=np.uint16)
    lo = np.zeros_like(hi)
    if rows > 0 and k > 0:
        hi = np.zeros((rows, k), dtype=np.uint16)
        lo = np.zeros_like(hi)
        lib().oracle_split_rows(rows, k, _ptr(X), sr, sp, _ptr(e), _ptr(hi), _ptr(lo))
    return e[:rows], hi[:rows, :k], lo[:rows, :k]


def split_rows3(X: np.ndarray, rows: int, k: int, sr: int, sp: int):
    """(e, hi, mid, lo3): the three-part split; hi and mid equal split_rows' hi and lo."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    e = np.zeros(max(rows, 1), dtype=np.int32)
    hi = np.zeros((max(rows, 1), max(k, 1)), dtype=np.uint16)
    mid = np.zeros_like(hi)
    lo3 = np.zeros_like(hi)
    if rows > 0 and k > 0:
        lib().oracle_split_rows3(rows, k, _ptr(X), sr, sp, _ptr(e), _ptr(hi), _ptr(mid), _ptr(lo3))
    return e[:rows], hi[:rows, :k], mid[:rows, :k], lo3[:rows, :k]


def split_third(x: float) -> int:
    return int(lib().oracle_split_third(float(x)))


def split3_exhaustive(u0: int = 0, u1: int = 1 << 32, nthreads: int = 0) -> np.ndarray:
    counts = np.zeros(3, dtype=np.int64)
    lib().oracle_split3_exhaustive(u0, u1, _ptr(counts), int(nthreads))
    return counts


def split_operand3(which: str, trans: str, rows_op: int, k: int, X: np.ndarray, ld: int):
    """(e, hi, mid, lo3) of op(A) rows (which='A') or op(B) columns (which='B')."""
    t = lib().oracle_trans_code(trans.encode())
    if t < 0:
        raise ValueError("bad transpose flag")
    if which == "A":
        sr, sp = (ld, 1) if t else (1, ld)
    else:
        sr, sp = (1, ld) if t else (ld, 1)
    return split_rows3(X, rows_op, k, sr, sp)


def split_operand(which: str, trans: str, rows_op: int, k: int, X: np.ndarray, ld: int):
    """(e, hi, lo) of op(A) rows (which='A') or op(B) columns (which='B')."""
    t = lib().oracle_trans_code(trans.encode())
    if t < 0:
        raise ValueError("bad transpose flag")
    if which == "A":
        sr, sp = (ld, 1) if t else (1, ld)      # opA(i,p) = A[i + p*lda] or A[p + i*lda]
    else:
        sr, sp = (1, ld) if t else (ld, 1)      # opB(p,j) = B[p + j*ldb] or B[j + p*ldb]
    return split_rows(X, rows_op, k, sr, sp)


def split_exhaustive(u0: int = 0, u1: int = 1 << 32, nthreads: int = 0) -> np.ndarray:
    counts = np.zeros(8, dtype=np.int64)
    lib().oracle_split_exhaustive(u0, u1, _ptr(counts), int(nthreads))
    return counts


def error_ratio(c_gpu: np.ndarray, c64: np.ndarray, bound: np.ndarray) -> float:
    """max_ij |c_gpu - c64| / bound; entries with bound 0 must match exactly (else inf)."""
    d = np.abs(c_gpu.astype(np.float64) - c64)
    zero = bound == 0
    if np.any(zero & (d != 0)):
        return float("inf")
    if d.size == 0:
        return 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(zero, 0.0, d / np.where(zero, 1.0, bound))
    if np.any(np.isnan(r)):
        return float("inf")
    return float(r.max())


def freivalds_ratio(opA, opB, C_in, C_out, alpha, beta, x):
    """Freivalds check of a full output, O(mk + kn + mn) per vector.

    ``opA`` (m x k), ``opB`` (k x n), ``C_in`` and ``C_out`` (m x n) are the
    logical matrices.  With y = C_out x and exact z = alpha opA (opB x) +
    beta C_in x, the componentwise bound |C_out - C_exact|_ij <= b_ij gives
      |y - z|_i <= sum_j b_ij |x_j|
                = 2 max(k,1) 2^-24 (|alpha| |opA| (|opB| |x|) + |beta| |C_in| |x|)_i .
    Everything is evaluated in float64; the float64 evaluation error of y and
    z (relative about (k + n) 2^-53) is added to the allowance.  Returns the
    max over rows of |y - z| / allowance.
    """
    m, k = opA.shape
    n = opB.shape[1]
    A64, B64 = opA.astype(np.float64), opB.astype(np.float64)
    Cin, Cout = C_in.astype(np.float64), C_out.astype(np.float64)
    x = x.astype(np.float64)
    ax = np.abs(x)
    use_ab = alpha != 0 and k > 0
    y = Cout @ x
    z = np.zeros(m)
    absterm = np.zeros(m)
    if use_ab:
        z += alpha * (A64 @ (B64 @ x))
        absterm += abs(alpha) * (np.abs(A64) @ (np.abs(B64) @ ax))
    if beta != 0:
        z += beta * (Cin @ x)
        absterm += abs(beta) * (np.abs(Cin) @ ax)
    allow = 2.0 * max(k, 1) * 2.0**-24 * absterm + 4.0 * (k + n + 2) * 2.0**-53 * (absterm + np.abs(Cout) @ ax)
    d = np.abs(y - z)
    zero = allow == 0
    if np.any(zero & (d != 0)) or np.any(np.isnan(d)):
        return float("inf")
    r = np.where(zero, 0.0, d / np.where(zero, 1.0, allow))
    return float(r.max()) if r.size else 0.0
