"""Host logic of the grouped plans' panel ring (no GPU): regions of
increasing problems are placed one after another in a ring smaller than L2,
and a problem may only be packed once every earlier problem whose bytes it
overwrites has been read.  Checked against a byte-level replay of the ring
on random region sizes."""

import numpy as np
import pytest

from paper_1608_05265_gb300 import build, gbgemm


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return gbgemm.lib()


def replay(sizes, ring, offs):
    """Every earlier region overlapping each region, by direct interval tests."""
    over = []
    for i, (o, s) in enumerate(zip(offs, sizes)):
        over.append({j for j in range(i) if offs[j] < o + s and o < offs[j] + sizes[j]})
    return over


@pytest.mark.parametrize("seed", range(6))
def test_ring_waits_cover_every_overwritten_region(seed):
    rng = np.random.default_rng(seed)
    gran = 4096
    ring = gran * int(rng.integers(40, 200))
    n = 300
    sizes = [gran * int(x) for x in np.minimum(rng.geometric(0.15, n), ring // gran)]
    offs, waits = gbgemm.grouped_ring_layout(sizes, ring, gran)
    over = replay(sizes, ring, offs)
    guaranteed = []  # regions certainly read before region i is packed
    for i, (o, s) in enumerate(zip(offs, sizes)):
        assert o % gran == 0 and 0 <= o and o + s <= ring
        # placed right after the previous region, or at 0 when it did not fit
        if i > 0:
            nxt = offs[i - 1] + sizes[i - 1]
            assert o == (nxt if nxt + s <= ring else 0)
        # waits name earlier regions that really overlap, each once
        assert len(set(waits[i])) == len(waits[i])
        assert all(j < i and j in over[i] for j in waits[i])
        # a wait on j also covers what j waited for (j was packed after those were read)
        g = set(waits[i])
        for j in waits[i]:
            g |= guaranteed[j]
        guaranteed.append(g)
        assert over[i] <= g, (i, sorted(over[i] - g))


def test_batch_that_fits_waits_for_nothing():
    gran = 4096
    sizes = [gran * k for k in (1, 5, 3, 8, 2)]
    offs, waits = gbgemm.grouped_ring_layout(sizes, sum(sizes), gran)
    assert offs == [0, 4096, 6 * 4096, 9 * 4096, 17 * 4096]
    assert all(w == [] for w in waits)


def test_wrap_and_small_example():
    # ring of 10 granules; regions 4, 4, 4 (wraps), 6, 3
    gran = 4096
    sizes = [4 * gran, 4 * gran, 4 * gran, 6 * gran, 3 * gran]
    offs, waits = gbgemm.grouped_ring_layout(sizes, 10 * gran, gran)
    assert [o // gran for o in offs] == [0, 4, 0, 4, 0]
    assert waits == [[], [], [0], [1], [2]]


def test_bad_arguments():
    with pytest.raises(gbgemm.GbgemmError):
        gbgemm.grouped_ring_layout([4096, 5000], 1 << 20, 4096)   # not a multiple of the granule
    with pytest.raises(gbgemm.GbgemmError):
        gbgemm.grouped_ring_layout([1 << 21], 1 << 20, 4096)      # larger than the ring
