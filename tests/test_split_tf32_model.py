"""The error model behind the split-TF32 tolerance (CPU, no GPU).

Split TF32 stores each FP32 operand x as hi = tf32(x) and lo = tf32(x - hi), with tf32()
rounding to 10 mantissa bits, nearest with ties away from zero (the rounding the
operand pack uses), and forms a product as hi_a hi_b + hi_a lo_b + lo_a hi_b. The dropped
lo_a lo_b term and the rounding of the low parts are each about 2^-22 of |a b|, so a
product is off by at most ~2^-20 of its magnitude, and sums of products by that fraction
of the summed magnitudes: the basis of the 1e-5 tolerance the GPU tests hold split-TF32
sessions to. Here the model is evaluated exactly in FP64 on random operands over many
binades.
"""

import numpy as np


def tf32(x):
    """Round FP32 values to TF32 (10 explicit mantissa bits), nearest, ties away from zero."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & ~np.uint64(0x1FFF)  # add half of the dropped 13 bits to the magnitude
    return b.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    hi = tf32(x)
    lo = tf32((x - hi).astype(np.float32))  # x - hi is exact in FP32
    return hi, lo


def test_tf32_rounding_keeps_ten_mantissa_bits():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(100000) * np.exp2(rng.integers(-40, 40, 100000))).astype(np.float32)
    t = tf32(x)
    assert np.all(t.view(np.uint32) & 0x1FFF == 0)
    rel = np.abs(t.astype(np.float64) - x) / np.abs(x.astype(np.float64))
    assert rel.max() <= 2.0 ** -11  # half a unit of the 11-bit significand
    # ties go away from zero
    one_and_half_ulp = np.float32(1.0 + 2.0 ** -11)
    assert tf32(one_and_half_ulp) == np.float32(1.0 + 2.0 ** -10)
    assert tf32(-one_and_half_ulp) == -np.float32(1.0 + 2.0 ** -10)


def test_split_products_are_fp32_class():
    rng = np.random.default_rng(2)
    n = 200000
    a = (rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))).astype(np.float32)
    b = (rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))).astype(np.float32)
    ah, al = split(a)
    bh, bl = split(b)
    f = lambda v: v.astype(np.float64)
    exact = f(a) * f(b)
    three = f(ah) * f(bh) + f(ah) * f(bl) + f(al) * f(bh)
    one = f(tf32(a)) * f(tf32(b))
    rel3 = np.abs(three - exact) / np.abs(exact)
    rel1 = np.abs(one - exact) / np.abs(exact)
    assert rel3.max() <= 2.0 ** -20
    assert rel1.max() > 2.0 ** -12  # a single TF32 product is ~2^-11: the split gains ~10 bits
    # a window's sum of products (the CSD sums): off by at most 2^-20 of the summed magnitudes
    K = 200
    A = a[: 1000 * K].reshape(1000, K)
    Bm = b[: 1000 * K].reshape(1000, K)
    Ah, Al = split(A)
    Bh, Bl = split(Bm)
    s_exact = np.sum(f(A) * f(Bm), axis=1)
    s3 = np.sum(f(Ah) * f(Bh) + f(Ah) * f(Bl) + f(Al) * f(Bh), axis=1)
    mag = np.sum(np.abs(f(A) * f(Bm)), axis=1)
    assert np.all(np.abs(s3 - s_exact) <= 2.0 ** -20 * mag)
