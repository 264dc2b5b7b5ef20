"""Pins of the oracle's point generator (step a1): Philox4x32-10 against the
published known-answer vectors, the counter layout and the uniform maps."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_sample_word_layout():
    # coordinate j of sample i draws word j%4 of block (j//4, i lo, i hi, sid), key (seed, job)
    seed, job, sid, d = 7, 3, 11, 10
    for i in (0, 1, 12345, (5 << 32) + 17):
        w = oracle.sample_words(seed, job, sid, i, d)
        for j in range(d):
            blk = oracle.philox4x32_10([j // 4, i & 0xFFFFFFFF, i >> 32, sid], [seed, job])
            assert w[j] == blk[j % 4]


def test_streams_differ_by_every_counter_field():
    base = oracle.sample_words(1, 0, 0, 0, 8)
    assert not np.array_equal(base, oracle.sample_words(2, 0, 0, 0, 8))
    assert not np.array_equal(base, oracle.sample_words(1, 1, 0, 0, 8))
    assert not np.array_equal(base, oracle.sample_words(1, 0, 1, 0, 8))
    assert not np.array_equal(base, oracle.sample_words(1, 0, 0, 1, 8))
    assert not np.array_equal(base, oracle.sample_words(1, 0, 0, 1 << 32, 8))


def test_points_inside_box_and_uniform():
    d = 4
    lo = np.array([-5.0, 0.0, -1.0, 2.0])
    hi = np.array([5.0, 5.0, 3.0, 2.5])
    for fp32 in (False, True):
        y = oracle.points(d, lo, hi, sid=0, seed=1, job_id=0, first=0, count=200000,
                          fp32_points=fp32)
        assert np.all(y >= lo) and np.all(y <= hi)
        u = (y - lo) / (hi - lo)
        # mean 1/2 and variance 1/12 of U(0,1), 200k draws: 6-sigma bands
        assert np.all(np.abs(u.mean(axis=0) - 0.5) < 6 * np.sqrt(1 / 12 / 2e5))
        assert np.all(np.abs(u.var(axis=0) - 1 / 12) < 6 * np.sqrt(1 / 180 / 2e5))


def test_fp32_points_are_floats_and_close_to_fp64_points():
    d = 20
    lo, hi = np.full(d, -5.0), np.full(d, 5.0)
    y64 = oracle.points(d, lo, hi, 3, 2, 0, 0, 1000, fp32_points=False)
    y32 = oracle.points(d, lo, hi, 3, 2, 0, 0, 1000, fp32_points=True)
    assert np.array_equal(y32.astype(np.float32).astype(np.float64), y32)
    # the FP32 grid is 2^-23 of the width; the FP64 one 2^-32
    assert np.max(np.abs(y32 - y64)) <= 10.0 * 2.0 ** -23 + 5.0 * 2.0 ** -24


def test_uniform_map_endpoints():
    # word 0 and word 2^32-1 map to the first and last grid midpoints, never to lo or hi
    lo, hi = np.zeros(1), np.ones(1)
    # find the words of sample 0 and check the map against them directly
    w = oracle.sample_words(9, 0, 0, 0, 1)[0]
    y = oracle.points(1, lo, hi, 0, 9, 0, 0, 1)[0, 0]
    assert y == (float(w) + 0.5) * 2.0 ** -32
    y32 = oracle.points(1, lo, hi, 0, 9, 0, 0, 1, fp32_points=True)[0, 0]
    assert y32 == ((int(w) >> 9) + 0.5) * 2.0 ** -23
