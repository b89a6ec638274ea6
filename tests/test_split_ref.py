"""Pins of the oracle's hi/lo BF16 split and power-of-two row scaling.

The split is the precision-recovery step of the tensor path (each FP32
operand x becomes hi + lo, two BF16 values; three BF16 products recover FP32
accuracy).  The oracle restates it from the IEEE-754 definitions; these tests
pin that restatement to facts that do not come from it:
  * BF16 round-to-nearest-even against torch's CPU float->bfloat16 cast;
  * worked values computed by hand (ties to even, carries into the exponent);
  * the frexp exponent against Python's math.frexp;
  * an exhaustive scan of all 2^32 float patterns for the invariants
    (x - hi exact in float, |x - hi - lo| <= 2^-17 |x| for |x| >= 2^-100,
    sign kept, overflow to Inf exactly at 2^128 (1 - 2^-9), lo = 0 for
    non-finite x).
"""

import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1608_05265_gb300 import synth


def f32(bits):
    return float(np.array([bits], dtype=np.uint32).view(np.float32)[0])


def test_bf16_rne_matches_torch_on_sample():
    rng = np.random.default_rng(0)
    bits = np.concatenate([
        np.arange(0, 1 << 32, 65521, dtype=np.uint64),          # strided sweep
        rng.integers(0, 1 << 32, 200000, dtype=np.uint64),     # random patterns
        np.array([0x3F808000, 0x3F818000, 0x3F80FFFF, 0x7F7F8000, 0x7F7F7FFF, 0x00008000,
                  0x00018000, 0x80008000, 0x7F800000, 0xFF800000, 0x00000001], dtype=np.uint64),
    ]).astype(np.uint32)
    x = bits.view(np.float32)
    t = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    lib = O.lib()
    got = np.array([lib.oracle_bf16_rne(float(v)) for v in x[:: 7]], dtype=np.uint16)
    want = t[:: 7]
    nan = np.isnan(x[:: 7])
    assert np.array_equal(got[~nan], want[~nan])
    gotf = np.array(got, dtype=np.uint32) << 16
    assert np.all(np.isnan(gotf.view(np.float32)[nan]))


@pytest.mark.parametrize("x,hi,lo", [
    (1.0, 0x3F80, 0x0000),
    (1.0 + 2.0**-8, 0x3F80, 0x3B80),           # exact tie -> even (1.0); remainder 2^-8
    (1.0 + 3 * 2.0**-8, 0x3F82, 0xBB80),       # tie between 1+2^-7 and 1+2^-6 -> even 1+2^-6
    (1.0 + 2.0**-8 + 2.0**-12, 0x3F81, 0xBB70),  # above the tie -> up; lo = -(2^-8 - 2^-12) = -1.875*2^-9
    (-2.5, 0xC020, 0x0000),
    (2.0 - 2.0**-23, 0x4000, 0xB400),          # carries into the exponent; lo = -2^-23
    (float("inf"), 0x7F80, 0x0000),
])
def test_split_worked_values(x, hi, lo):
    e, H, L = O.split_rows(np.array([x], dtype=np.float32), 1, 1, 1, 1)
    if math.isfinite(x):
        # a single-element row is scaled to [0.5, 1): compare on the unscaled split
        h = O.bf16_rne(x)
        assert h == hi
        r = np.float32(x) - np.array([h << 16], dtype=np.uint32).view(np.float32)[0]
        assert O.bf16_rne(float(r)) == lo
    else:
        assert (int(H[0, 0]), int(L[0, 0])) == (hi, lo)


def test_scale_exponent_matches_frexp_outside_the_well_scaled_band():
    # badly scaled maxima (outside [2^-48, 2^48)) take the frexp exponent
    vals = [1e-30, 3.4e38, f32(0x00000001), f32(0x007FFFFF), f32(0x00800000), 2.0**-127,
            2.0**48, 2.0**-48 * (1 - 2.0**-24), 1e20]
    for v in vals:
        assert O.scale_exponent(v) == math.frexp(float(np.float32(v)))[1], v
    # well scaled maxima are not scaled
    for v in [1.0, 0.5, 0.75, 3.0, 2.0**-48, 2.0**48 * (1 - 2.0**-24), 1e-14, 1e14]:
        assert O.scale_exponent(v) == 0, v
    assert O.scale_exponent(0.0) == 0
    assert O.scale_exponent(float("inf")) == 0
    assert O.scale_exponent(float("nan")) == 0


def test_split_rows_reconstructs_and_normalises():
    rows, k = 16, 300
    X = synth.normal_rowscaled_matrix(4, 0, rows, k, rows, elo=-120, ehi=120)
    e, hi, lo = O.split_rows(X, rows, k, 1, rows)
    L = synth.logical(X, rows, k, rows).astype(np.float64)
    hf = (hi.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    lf = (lo.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    scaled = 0
    for r in range(rows):
        amax = np.abs(L[r]).max()
        if 2.0**-48 <= amax < 2.0**48:
            assert e[r] == 0
        else:
            assert e[r] == math.frexp(amax)[1]
            scaled += 1
        xs = L[r] * 2.0 ** (-int(e[r]))
        if e[r] != 0:
            assert 0.5 <= np.abs(xs).max() < 1.0
        big = np.abs(xs) >= 2.0**-100
        assert np.all(np.abs(xs - hf[r] - lf[r])[big] <= 2.0**-17 * np.abs(xs)[big])
    assert 0 < scaled < rows


def test_split_operand_layouts_agree():
    m, k = 19, 37
    A_n = synth.uniform_matrix(5, 0, m, k, m + 3)
    L = synth.logical(A_n, m, k, m + 3)
    A_t = synth.place_colmajor(L.reshape(-1), k, m, k + 5)  # stored k x m, op = transpose
    a = O.split_operand("A", "N", m, k, A_n, m + 3)
    b = O.split_operand("A", "T", m, k, A_t, k + 5)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # op(B) columns: B stored k x n (N) vs n x k (T)
    n = m
    B_n = synth.place_colmajor(L.reshape(-1), k, n, k + 1)    # B[p + j*ldb] = opB(p, j) = L[j, p]
    B_t = synth.place_colmajor(L.T.reshape(-1), n, k, n + 2)  # B[j + p*ldb] = opB(p, j) = L[j, p]
    c = O.split_operand("B", "N", n, k, B_n, k + 1)
    d = O.split_operand("B", "T", n, k, B_t, n + 2)
    for x, y, z in zip(a, c, d):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_split_scaling_handles_extremes():
    # Rows near FLT_MAX and near the bottom of the normal range: the unscaled
    # split overflows hi (near FLT_MAX) or leaves lo below the normal range;
    # after scaling both are ordinary.
    row_big = np.array([3.4e38, -1.0e38, 2.0e37], dtype=np.float32)
    e, hi, lo = O.split_rows(row_big, 1, 3, 3, 1)
    hf = (hi.astype(np.uint32) << 16).view(np.float32)
    assert np.all(np.isfinite(hf)) and e[0] == 128
    assert O.bf16_rne(3.4e38) == 0x7F80  # unscaled: above 2^128 (1 - 2^-9), rounds to Inf
    row_small = np.array([1.5e-38, -3e-39, 7e-39], dtype=np.float32)
    e, hi, lo = O.split_rows(row_small, 1, 3, 3, 1)
    lf = (lo.astype(np.uint32) << 16).view(np.float32)
    assert e[0] == math.frexp(float(np.float32(1.5e-38)))[1]
    assert np.all(np.abs(lf[lf != 0]) >= 2.0**-126)


def test_split_exhaustive_invariants():
    c = O.split_exhaustive()
    assert c[0] == (1 << 32) - 2 * (1 << 23)  # every pattern whose exponent field is not all ones
    assert list(c[1:7]) == [0, 0, 0, 0, 0, 0]
    assert c[7] <= 2**23  # max relative residual <= 2^-17


@pytest.mark.parametrize("x", [1.0 + 2.0**-8 + 2.0**-12 + 2.0**-20, -3.14159265, 1.0 / 3.0, 2.0**-90 * 1.2345,
                               float(np.float32(1e30)), 0.1])
def test_three_part_split_is_exact(x):
    x = float(np.float32(x))
    h = O.bf16_rne(x)
    hf = float(np.array([h << 16], dtype=np.uint32).view(np.float32)[0])
    r1 = float(np.float32(x) - np.float32(hf))
    m = O.bf16_rne(r1)
    mf = float(np.array([m << 16], dtype=np.uint32).view(np.float32)[0])
    lo = O.split_third(x)
    lf = float(np.array([lo << 16], dtype=np.uint32).view(np.float32)[0])
    assert hf + mf + lf == x  # exact in double
    # the third part is a BF16 rounding of an exact float remainder
    assert lo == O.bf16_rne(float(np.float32(r1) - np.float32(mf)))


def test_three_part_split_exhaustive():
    c = O.split3_exhaustive()
    assert c[0] > 3_000_000_000
    assert c[1] == 0 and c[2] == 0


def test_split_rows3_matches_two_part_split():
    rows, k = 9, 77
    X = synth.normal_rowscaled_matrix(6, 0, rows, k, rows, elo=-70, ehi=70)
    e, hi, lo = O.split_rows(X, rows, k, 1, rows)
    e3, hi3, mid3, lo3 = O.split_rows3(X, rows, k, 1, rows)
    assert np.array_equal(e, e3) and np.array_equal(hi, hi3) and np.array_equal(lo, mid3)
    L = synth.logical(X, rows, k, rows).astype(np.float64)
    f = lambda a: (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)  # noqa: E731
    xs = L * np.ldexp(1.0, -e3.astype(np.int64))[:, None]
    big = np.abs(xs) >= 2.0**-100
    assert np.array_equal((f(hi3) + f(mid3) + f(lo3))[big], xs[big])
