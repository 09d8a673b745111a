"""Pins for the oracle's counter-based random numbers (reading R-rng).

The paper names no generator (Sec. 4.2.2 only asks for one state per thread);
the reading is Philox4x32-10, pinned here by published known-answer vectors.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    got = O.philox4x32_10(ctr, key)
    assert [int(x) for x in got] == want


def test_uniform_open_interval_and_float_exact():
    xs = [0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFE00, 0xFFFFFFFF]
    for x in xs:
        u = O.uniform01(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exact in float, so both sides see the same r
    assert O.uniform01(0) == 2.0 ** -24
    assert O.uniform01(0xFFFFFFFF) == 1.0 - 2.0 ** -24


def test_uniform_is_uniform():
    rng = np.random.Generator(np.random.PCG64(5))
    words = rng.integers(0, 2 ** 32, size=20000, dtype=np.uint64)
    u = np.array([O.uniform01(int(w)) for w in words])
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_streams_select_words_of_one_philox_call():
    seed = 0x1234_5678_9ABC_DEF0
    key = [seed & 0xFFFFFFFF, seed >> 32]
    # start node: word 0 of counter (0xFFFFFFFF, 0, ant, it)
    out = O.philox4x32_10([0xFFFFFFFF, 0, 7, 3], key)
    assert O.word_start(seed, 3, 7) == out[0]
    # candidate slot s at step t: word t%4 of (s, t//4, ant, it)
    for t in range(1, 9):
        out = O.philox4x32_10([5, t >> 2, 7, 3], key)
        assert O.word_cand(seed, 3, 7, t, 5) == out[t & 3]
    # whole-row node v at step t: word v%4 of (2^31 | v//4, t, ant, it)
    for v in range(0, 9):
        out = O.philox4x32_10([0x80000000 | (v >> 2), 4, 7, 3], key)
        assert O.word_row(seed, 3, 7, 4, v) == out[v & 3]


def test_start_node_uniform():
    n = 13
    seed = 42
    counts = np.zeros(n)
    for it in range(200):
        for ant in range(50):
            s = O.start_node(seed, it, ant, n)
            assert 0 <= s < n
            counts[s] += 1
    assert stats.chisquare(counts).pvalue > 1e-3


def test_start_node_is_multiply_shift():
    for (it, ant, n) in [(0, 0, 1000), (5, 17, 3), (99, 999, 65535)]:
        x = O.word_start(9, it, ant)
        assert O.start_node(9, it, ant, n) == (x * n) >> 32
