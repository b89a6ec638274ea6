"""Seeded synthetic inputs for sgemm workloads.

This module is shared by the tests, the benchmark and the CPU oracle's callers.
It holds no GEMM arithmetic: it only draws numbers and lays them out in
column-major storage with leading-dimension padding.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in its counter form: the
i-th output of a stream with base state ``s`` is ``mix(s + (i + 1) * GAMMA)``,
so any element can be drawn independently and the whole fill vectorises.

Distributions:
  * uniform[-1, 1):  ``(u >> 40) * 2**-23 - 1``; every value is an exact float.
  * normal(0, 1):    Box-Muller (cosine branch) in double from two draws,
                     rounded to float.
  * integer e in [lo, hi]: ``lo + (u >> 32) % (hi - lo + 1)``.

Matrices are column-major.  An ``rows x cols`` matrix with leading dimension
``ld >= rows`` is stored as ``cols`` columns of ``ld`` floats.  Element
``(r, c)`` takes draw number ``c * rows + r`` of its stream, so the fill runs
column by column over the logical rows only.  Padding rows ``rows <= r < ld``
hold the NaN sentinel ``SENTINEL_BITS`` and are never drawn, which lets a test
see any read or write outside the logical matrix.
"""

from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: Quiet-NaN bit pattern written into every padding slot of a generated matrix.
SENTINEL_BITS = 0x7FC0FFEE


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_base(seed: int, stream: int) -> np.uint64:
    """Base state of sub-stream ``stream`` of ``seed`` (draw ``stream`` of the seed's own stream)."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(stream + 1) * GAMMA
        return _mix(np.array([s], dtype=np.uint64))[0]


def draws(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` raw 64-bit draws of a sub-stream, starting at draw ``offset``."""
    base = stream_base(seed, stream)
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(base + idx * GAMMA)


def uniform_pm1(u: np.ndarray) -> np.ndarray:
    """Map raw draws to exact floats in [-1, 1)."""
    q = (u >> np.uint64(40)).astype(np.int64) - (1 << 23)
    return (q.astype(np.float64) * 2.0**-23).astype(np.float32)


def normal01(u: np.ndarray) -> np.ndarray:
    """Map pairs of raw draws (even, odd) to normal(0,1) floats by Box-Muller."""
    a = u[0::2]
    b = u[1::2]
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0**-53
    u2 = (b >> np.uint64(11)).astype(np.float64) * 2.0**-53
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return z.astype(np.float32)


def int_range(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    return (lo + ((u >> np.uint64(32)) % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int64)


def sentinel_f32() -> np.float32:
    return np.array([SENTINEL_BITS], dtype=np.uint32).view(np.float32)[0]


def place_colmajor(vals_by_col: np.ndarray, rows: int, cols: int, ld: int) -> np.ndarray:
    """Lay ``rows*cols`` values (column by column) into ``cols`` columns of ``ld`` floats.

    Returns a flat float32 array of ``ld * cols`` elements (at least one element
    so that an empty matrix still has an address).
    """
    if ld < max(1, rows):
        raise ValueError("ld < rows")
    out = np.empty((cols, ld), dtype=np.float32)
    out.view(np.uint32)[:] = SENTINEL_BITS
    if rows > 0 and cols > 0:
        out[:, :rows] = vals_by_col.reshape(cols, rows)
    flat = out.reshape(-1)
    if flat.size == 0:
        flat = np.full(1, sentinel_f32(), dtype=np.float32)
    return flat


def uniform_block(seed: int, stream: int, rows: int, r0: int, r1: int, c0: int, c1: int) -> np.ndarray:
    """Rows r0..r1-1, columns c0..c1-1 of the uniform matrix of ``rows`` rows
    drawn by ``uniform_matrix(seed, stream, rows, ...)``, as a column-major
    block with leading dimension r1 - r0 (flat float32 array)."""
    r = np.arange(r0, r1, dtype=np.uint64)
    c = np.arange(c0, c1, dtype=np.uint64)
    idx = (c[:, None] * np.uint64(rows) + r[None, :]).reshape(-1)
    base = stream_base(seed, stream)
    with np.errstate(over="ignore"):
        u = _mix(base + (idx + np.uint64(1)) * GAMMA)
    return uniform_pm1(u)


def uniform_matrix(seed: int, stream: int, rows: int, cols: int, ld: int) -> np.ndarray:
    v = uniform_pm1(draws(seed, stream, rows * cols))
    return place_colmajor(v, rows, cols, ld)


def normal_rowscaled_matrix(seed: int, stream: int, rows: int, cols: int, ld: int,
                            elo: int = -20, ehi: int = 20) -> np.ndarray:
    """normal(0,1) entries times 2**e_r, one integer e_r in [elo, ehi] per row.

    Sub-stream ``stream`` gives the values (two draws per entry), sub-stream
    ``stream + 1`` the row exponents.
    """
    e = int_range(draws(seed, stream + 1, rows), elo, ehi)
    scale = np.ldexp(np.ones(rows, dtype=np.float32), e.astype(np.int32)).astype(np.float32)
    if ld < max(1, rows):
        raise ValueError("ld < rows")
    out = np.empty((cols, ld), dtype=np.float32)
    out.view(np.uint32)[:] = SENTINEL_BITS
    # column blocks of at most 2^24 entries keep the temporaries small; column c
    # takes draws 2 c rows .. 2 (c + 1) rows - 1 either way
    step = max(1, (1 << 24) // max(rows, 1))
    for c0 in range(0, cols if rows > 0 else 0, step):
        c1 = min(cols, c0 + step)
        v = normal01(draws(seed, stream, 2 * rows * (c1 - c0), offset=2 * rows * c0)).reshape(c1 - c0, rows)
        out[c0:c1, :rows] = v * scale[None, :]
    flat = out.reshape(-1)
    if flat.size == 0:
        flat = np.full(1, sentinel_f32(), dtype=np.float32)
    return flat


def small_int_matrix(seed: int, stream: int, rows: int, cols: int, ld: int, lo: int = -4, hi: int = 4) -> np.ndarray:
    v = int_range(draws(seed, stream, rows * cols), lo, hi).astype(np.float32)
    return place_colmajor(v, rows, cols, ld)


def logical(flat: np.ndarray, rows: int, cols: int, ld: int) -> np.ndarray:
    """The ``rows x cols`` logical matrix (as a float array indexed [r, c]) of a column-major buffer."""
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols), dtype=flat.dtype)
    return flat[: ld * cols].reshape(cols, ld)[:, :rows].T


def padding_is_sentinel(flat: np.ndarray, rows: int, cols: int, ld: int) -> bool:
    """True when every padding slot (rows <= r < ld) still holds the sentinel bits."""
    if cols == 0 or ld == rows:
        return True
    bits = flat[: ld * cols].view(np.uint32).reshape(cols, ld)[:, rows:]
    return bool(np.all(bits == SENTINEL_BITS))


# ----------------------------------------------------------------------------
# Workload recipes.  Stream numbers: A = 0, B = 2, C = 4 (each may use the next
# number for an auxiliary draw such as row exponents).
# ----------------------------------------------------------------------------

def op_shape(trans: str, rows_op: int, cols_op: int) -> tuple[int, int]:
    """Stored (rows, cols) of a matrix whose op() is rows_op x cols_op."""
    return (rows_op, cols_op) if trans in "Nn" else (cols_op, rows_op)


def gemm_problem(kind: str, seed: int, transa: str, transb: str, m: int, n: int, k: int,
                 pad: int = 0, lda: int | None = None, ldb: int | None = None, ldc: int | None = None):
    """Generate (A, lda, B, ldb, C, ldc) for one problem.

    ``kind`` is ``uniform`` (uniform[-1,1)), ``normal_rowscaled`` (normal(0,1)
    times 2**e per stored row, e in [-20, 20]) or ``smallint`` (integers in
    [-4, 4]).  Leading dimensions default to stored rows + ``pad``.
    """
    ar, ac = op_shape(transa, m, k)
    br, bc = op_shape(transb, k, n)
    lda = lda if lda is not None else max(1, ar + pad)
    ldb = ldb if ldb is not None else max(1, br + pad)
    ldc = ldc if ldc is not None else max(1, m + pad)
    if kind == "uniform":
        f = uniform_matrix
    elif kind == "normal_rowscaled":
        f = normal_rowscaled_matrix
    elif kind == "smallint":
        f = small_int_matrix
    else:
        raise ValueError(kind)
    A = f(seed, 0, ar, ac, lda)
    B = f(seed, 2, br, bc, ldb)
    C = f(seed, 4, m, n, ldc)
    return A, lda, B, ldb, C, ldc


def grouped_shapes(seed: int, count: int, lo: int = 16, hi: int = 1024):
    """Shapes and flags of a grouped batch.

    m, n, k = floor(exp(ln lo + u * (ln(hi+1) - ln lo))) with u uniform in [0,1),
    clamped to [lo, hi]; transa, transb uniform over {N, T}.  Sub-stream 10
    holds the shape draws (3 per problem, m then n then k), sub-stream 11 the
    flag draws (2 per problem).
    """
    u = draws(seed, 10, 3 * count)
    f = (u >> np.uint64(11)).astype(np.float64) * 2.0**-53
    dims = np.floor(np.exp(math.log(lo) + f * (math.log(hi + 1) - math.log(lo)))).astype(np.int64)
    dims = np.clip(dims, lo, hi).reshape(count, 3)
    fl = draws(seed, 11, 2 * count).reshape(count, 2)
    flags = np.where((fl >> np.uint64(63)) == 1, "T", "N")
    return [(str(flags[g, 0]), str(flags[g, 1]), int(dims[g, 0]), int(dims[g, 1]), int(dims[g, 2]))
            for g in range(count)]


def grouped_problem_data(seed: int, g: int, transa: str, transb: str, m: int, n: int, k: int):
    """Data of problem ``g`` of a grouped batch: tight leading dimensions, uniform[-1,1).

    Problem g draws from sub-streams 100 + 6g (A), 102 + 6g (B), 104 + 6g (C).
    """
    ar, ac = op_shape(transa, m, k)
    br, bc = op_shape(transb, k, n)
    lda, ldb, ldc = max(1, ar), max(1, br), max(1, m)
    A = uniform_matrix(seed, 100 + 6 * g, ar, ac, lda)
    B = uniform_matrix(seed, 102 + 6 * g, br, bc, ldb)
    C = uniform_matrix(seed, 104 + 6 * g, m, n, ldc)
    return A, lda, B, ldb, C, ldc
