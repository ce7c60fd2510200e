"""The digit decompositions behind the fixed-point forms, restated on the host.

Both forms hold a tensor as integers X (|X| < 2^b) and cut every integer into
balanced digits that the tensor cores take exactly (Ozaki et al., Numer.
Algorithms 59 (2012), error-free slicing).  These tests pin the arithmetic
facts the kernels rely on, for the extreme and random integers:

* FX32 (b = 31): x = d0 2^24 + d1 2^16 + d2 2^8 + d3 with d0 in [-128, 128] and
  d1..d3 in [-128, 127], read without a carry chain from y = x + 0x808080; the
  slices d_t 2^(-8t) are exact in bf16.
* FX32H (b = 29): x = d0 2^22 + d1 2^11 + d2 with d0 in [-128, 128] and d1, d2
  in [-1024, 1023], read from y = x + 0x200400; the slices d0 2^8, d1 2^-3,
  d2 2^-14 are exact, normal (or zero) fp16 values, and x = 2^14 (sum).
* Level 0 (the products of the leading digits) stays an exact FP32 sum in the
  accumulator for contraction lengths up to 1024 (both forms: |d0| <= 128).
"""
import numpy as np
import pytest

RNG = np.random.default_rng(2112)


def _ints(bits, n=20000):
    lim = (1 << bits) - 1
    edge = np.array([0, 1, -1, lim, -lim, lim - 1, -(lim - 1), 1 << (bits - 1), -(1 << (bits - 1)),
                     0x3FF, -0x3FF, 0x400, -0x400, 0x7FF, -0x7FF, 0x80, -0x80, 0xFF, -0xFF], dtype=np.int64)
    return np.concatenate([edge, RNG.integers(-lim, lim + 1, size=n, dtype=np.int64)])


def fx32h_digits(x):
    y = x + 0x200400                      # int32 arithmetic: no overflow below 2^29
    d0 = y >> 22                          # arithmetic shift
    d1 = ((y >> 11) & 0x7FF) - 1024
    d2 = (y & 0x7FF) - 1024
    return d0, d1, d2


def fx32_digits(x):
    y = x + 0x808080
    d0 = y >> 24
    d1 = ((y >> 16) & 0xFF) - 128
    d2 = ((y >> 8) & 0xFF) - 128
    d3 = (y & 0xFF) - 128
    return d0, d1, d2, d3


def test_fx32h_digits_reconstruct_and_are_balanced():
    x = _ints(29)
    assert np.all(np.abs(x + 0x200400) < 2 ** 31)
    d0, d1, d2 = fx32h_digits(x)
    assert np.array_equal(d0 * 2 ** 22 + d1 * 2 ** 11 + d2, x)
    assert d0.min() >= -128 and d0.max() <= 128
    assert d1.min() >= -1024 and d1.max() <= 1023
    assert d2.min() >= -1024 and d2.max() <= 1023


def test_fx32h_slices_are_exact_normal_fp16():
    x = _ints(29)
    d0, d1, d2 = fx32h_digits(x)
    tiny = np.finfo(np.float16).tiny      # smallest normal fp16, 2^-14
    total = np.zeros(x.shape, dtype=np.float64)
    for d, sc in ((d0, 2.0 ** 8), (d1, 2.0 ** -3), (d2, 2.0 ** -14)):
        v = d.astype(np.float64) * sc
        h = v.astype(np.float16)
        assert np.array_equal(h.astype(np.float64), v)          # exact
        nz = v != 0
        assert np.all(np.abs(v[nz]) >= tiny)                     # normal
        assert np.all(np.abs(v) <= 2.0 ** 15)                    # in range
        total += v
    assert np.array_equal(total * 2.0 ** 14, x.astype(np.float64))


def test_fx32_digits_reconstruct_and_slices_are_exact_bf16():
    x = _ints(31)
    d = fx32_digits(x)
    assert np.array_equal(d[0] * 2 ** 24 + d[1] * 2 ** 16 + d[2] * 2 ** 8 + d[3], x)
    assert d[0].min() >= -128 and d[0].max() <= 128
    for t in (1, 2, 3):
        assert d[t].min() >= -128 and d[t].max() <= 127
    # bf16 keeps 8 significant bits: every digit (|d| <= 128) times a power of two is exact
    for t in range(4):
        v = (d[t].astype(np.float64) * 2.0 ** (-8 * t)).astype(np.float32)
        bits = v.view(np.uint32)
        assert np.all(bits & 0xFFFF == 0)


@pytest.mark.parametrize("K", [1, 256, 1024])
def test_level0_sums_are_exact_in_fp32(K):
    """The level-0 accumulator sums K products of leading digits (|d0| <= 128);
    in units of the product's scale the partial sums stay integers below 2^24,
    so FP32 accumulation in any order is exact."""
    d0a = RNG.integers(-128, 129, size=(8, K))
    d0b = RNG.integers(-128, 129, size=(8, K))
    d0a[0] = 128
    d0b[0] = 128                          # the worst case: all products 2^14
    exact = (d0a * d0b).sum(axis=1)
    acc = np.zeros(8, dtype=np.float32)
    for k in range(K):
        acc = (acc + (d0a[:, k] * d0b[:, k]).astype(np.float32)).astype(np.float32)
    assert np.array_equal(acc.astype(np.int64), exact)
    assert np.abs(exact).max() <= K * 2 ** 14 <= 2 ** 24
