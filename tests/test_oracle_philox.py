"""Pins for the oracle's Philox4x32-10 + Box-Muller sketch generator."""

import os

import numpy as np
import pytest
import scipy.stats

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    out = philox.philox4x32_10(np.array(ctr), np.array(key))
    assert [int(x) for x in out] == expect


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64)
    key = rng.integers(0, 2**32, size=(2,), dtype=np.uint64)
    batch = philox.philox4x32_10(ctr, key)
    for i in range(64):
        assert np.array_equal(batch[i], philox.philox4x32_10(ctr[i], key))


def test_gaussian_block_is_standard_normal():
    z = philox.gaussian_block(seed=123, t=4, j=9, rows=1000, cols=400).ravel()
    assert abs(z.mean()) < 5e-3
    assert abs(z.var() - 1.0) < 5e-3
    # Kolmogorov-Smirnov against the exact N(0,1) CDF (library, independent)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3


def test_gaussian_block_counter_addressing():
    # column-major linear index m = c*rows + k: a wider block extends a
    # narrower one, and the columns of an (r x c) block are the r-chunks of
    # one long column of length r*c.
    a = philox.gaussian_block(7, 3, 11, rows=37, cols=5)
    b = philox.gaussian_block(7, 3, 11, rows=37, cols=9)
    assert np.array_equal(a, b[:, :5])
    long = philox.gaussian_block(7, 3, 11, rows=37 * 9, cols=1)[:, 0]
    assert np.array_equal(b, long.reshape(9, 37).T)


def test_gaussian_block_streams_differ():
    base = philox.gaussian_block(1, 0, 0, 16, 4)
    for kw in [dict(seed=2, t=0, j=0), dict(seed=1, t=1, j=0), dict(seed=1, t=0, j=1)]:
        other = philox.gaussian_block(rows=16, cols=4, **kw)
        assert not np.allclose(base, other)
    other = philox.gaussian_block(1, 0, 0, 16, 4, stream=philox.STREAM_ADAPTIVE)
    assert not np.allclose(base, other)
    # the 64-bit seed uses both key words
    hi = philox.gaussian_block(1 + (1 << 32), 0, 0, 16, 4)
    assert not np.allclose(base, hi)


def test_box_muller_pairs_independent():
    z = philox.gaussian_block(99, 0, 0, rows=4, cols=100000)   # rows 0/1 are one pair
    c = np.corrcoef(z[0], z[1])[0, 1]
    assert abs(c) < 0.02
