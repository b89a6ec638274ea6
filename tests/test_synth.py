"""The seeded generator: SplitMix64 against its published outputs, exact
uniform values, sentinel padding, determinism."""

import numpy as np

from paper_1608_05265_gb300 import synth


def test_splitmix64_published_outputs():
    # SplitMix64 seeded with state 0 (Steele, Lea, Flood 2014): the first three
    # outputs, as listed with the reference implementation.
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    idx = np.arange(1, 4, dtype=np.uint64)
    with np.errstate(over="ignore"):
        got = synth._mix(idx * synth.GAMMA)
    assert [int(x) for x in got] == want


def test_uniform_exact_and_in_range():
    v = synth.uniform_pm1(synth.draws(0, 0, 100000))
    assert v.dtype == np.float32
    assert v.min() >= -1.0 and v.max() < 1.0
    q = v.astype(np.float64) * 2.0**23
    assert np.array_equal(q, np.round(q))
    assert abs(float(v.mean())) < 0.01


def test_normal_moments():
    v = synth.normal01(synth.draws(3, 0, 400000)).astype(np.float64)
    assert abs(v.mean()) < 0.01 and abs(v.std() - 1.0) < 0.01


def test_padding_sentinel_and_layout():
    A = synth.uniform_matrix(1, 0, 5, 3, 8)
    assert A.size == 24
    assert synth.padding_is_sentinel(A, 5, 3, 8)
    L = synth.logical(A, 5, 3, 8)
    assert L.shape == (5, 3) and np.all(np.isfinite(L))
    # element (r, c) is draw number c*rows + r
    d = synth.uniform_pm1(synth.draws(1, 0, 15))
    assert L[4, 2] == d[2 * 5 + 4]
    A[5] = 0.0
    assert not synth.padding_is_sentinel(A, 5, 3, 8)


def test_determinism_and_offset():
    a = synth.draws(42, 7, 1000)
    b = synth.draws(42, 7, 500, offset=500)
    assert np.array_equal(a[500:], b)
    assert not np.array_equal(synth.draws(42, 8, 10), a[:10])


def test_rowscaled_exponents_in_range():
    X = synth.normal_rowscaled_matrix(2, 0, 64, 200, 64)
    L = synth.logical(X, 64, 200, 64).astype(np.float64)
    amax = np.abs(L).max(axis=1)
    e = np.floor(np.log2(amax))
    assert e.min() >= -20 - 40 and e.max() <= 20 + 4
    assert e.max() - e.min() > 20


def test_grouped_shapes_range():
    s = synth.grouped_shapes(3, 4096)
    dims = np.array([x[2:] for x in s])
    assert dims.min() >= 16 and dims.max() <= 1024
    # log-uniform: the median is near sqrt(16*1025) ~ 128
    assert 100 < np.median(dims) < 165
    assert {x[0] for x in s} == {"N", "T"}


def test_uniform_block_matches_full_matrix():
    rows, cols, ld = 37, 23, 40
    full = synth.uniform_matrix(9, 2, rows, cols, ld)
    L = synth.logical(full, rows, cols, ld)
    blk = synth.uniform_block(9, 2, rows, 5, 30, 3, 20)
    assert np.array_equal(synth.logical(blk, 25, 17, 25), L[5:30, 3:20])
