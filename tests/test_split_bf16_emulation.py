"""CPU emulation (numpy) of the precision forms' products and their error.

The BF16 forms multiply FP32 operands on the tensor cores as BF16 with FP32
accumulation.  A single BF16 product rounds each operand to 8 significant
bits; the split form writes x = hi + lo with hi = bf16(x), lo = bf16(x - hi)
(x - hi is exact in FP32) and sums A_hi B_hi + A_hi B_lo + A_lo B_hi,
dropping only A_lo B_lo, so each operand carries about 16 bits.  This file
rounds to BF16 by round-to-nearest-even on the FP32 bit pattern, forms the
planes, and measures the relative error of both forms against FP64 on the
slice pass's product shapes (200 x 200 times 200 x l, Gaussian and
low-rank-plus-noise operands).  The split form's error sits below 1e-5 and
the single form's near 2e-3: the measured basis of the 1e-4 (split) and 1e-3
(single BF16) tolerances of the precision forms."""

import numpy as np
import pytest


def bf16(x):
    """Round FP32 values to BF16 (round to nearest, ties to even), as FP32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def planes(x):
    x = np.asarray(x, dtype=np.float32)
    hi = bf16(x)
    lo = bf16(x - hi)              # x - hi is exact in FP32
    return hi, lo


def test_bf16_rounding_known_values():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa (1) wins;
    # 1 + 3 * 2^-8 ties between 1 + 2^-7 and 1 + 2^-6: even (1 + 2^-6) wins
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20,
                  -2.5, 3.0e38], dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5])
    got = bf16(x).astype(np.float64)
    assert np.array_equal(got[:5], want)
    # 3e38 = 1.7632.. * 2^127 rounds to 226/128 * 2^127, within half a BF16 ulp
    assert got[5] == 226.0 / 128.0 * 2.0 ** 127
    assert abs(got[5] / float(x[5]) - 1) <= 2.0 ** -9
    hi, lo = planes(x[:4])
    assert np.all(np.abs((hi.astype(np.float64) + lo) - x[:4]) <= 2.0 ** -16 * np.abs(x[:4]))


def _products(A, B):
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    exact = A32.astype(np.float64) @ B32.astype(np.float64)
    Ah, Al = planes(A32)
    Bh, Bl = planes(B32)
    f = lambda X, Y: X.astype(np.float64) @ Y.astype(np.float64)   # products of BF16 values are exact in FP32
    single = f(Ah, Bh)
    split = f(Ah, Bh) + f(Ah, Bl) + f(Al, Bh)
    rel = lambda Z: np.linalg.norm(Z - exact) / np.linalg.norm(exact)
    return rel(single), rel(split)


@pytest.mark.parametrize("l", [20, 48])
@pytest.mark.parametrize("kind", ["gaussian", "lowrank"])
def test_split_form_carries_about_sixteen_bits(l, kind):
    rng = np.random.default_rng(l + (kind == "lowrank"))
    n = 200
    if kind == "gaussian":
        A = rng.standard_normal((n, n))
    else:
        A = rng.standard_normal((n, 10)) @ rng.standard_normal((10, n)) + 1e-3 * rng.standard_normal((n, n))
    B = np.linalg.qr(rng.standard_normal((n, l)))[0]      # an orthonormal panel, as Q or W
    e1, e3 = _products(A, B)
    assert e3 <= 1e-5
    assert 5e-4 <= e1 <= 5e-3
    assert e1 / e3 >= 100
