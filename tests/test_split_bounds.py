"""The error of the tensor-core forms' split products, emulated on the CPU.

An FP64 operand is rounded to FP32 (nearest) and split as x = hi + lo. The
split is BF16 hi and lo (nearest even; the form of opts.precision = 2) or TF32
hi and lo (nearest, ties away; opts.precision = 3). A product is then formed
as hi*hi + hi*lo + lo*hi.

The rank thresholds of those forms rest on the relative error of one such
product. The bounds follow from the split, with u_h the half-ulp of hi:
  BF16x3 (u_h = 2^-8): |x - hi - lo| <= u_h^2 |x|, and so is the dropped
    lo*lo, which gives at most 3 * 2^-16;
  3xTF32 (u_h = 2^-11): the same with u_h^2 = 2^-22, plus the FP32 rounding
    of each FP64 operand (2^-24), which gives at most 3 * 2^-22 + 2^-23 < 2^-20.
This test checks the bounds on random operands of mixed magnitude. It also
checks that they are tight within a factor of 8, so that a wrong rounding mode
or a dropped cross term (both plausible slips) fails it."""
from __future__ import annotations

import numpy as np


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def _bf16_rne(x32):
    """FP32 -> BF16 (kept as FP32): round to nearest, ties to even."""
    b = x32.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _tf32_rna(x32):
    """FP32 -> TF32 (kept as FP32): round to nearest, ties away from zero."""
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x1000) >> 13) << 13
    return r.astype(np.uint32).view(np.float32)


def _split(x64, rnd):
    x = _f32(x64)
    hi = rnd(x)
    lo = rnd((x - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def _product_rel_err(rnd, n=200000, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))
    y = rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))
    xh, xl = _split(x, rnd)
    yh, yl = _split(y, rnd)
    p = xh * yh + xh * yl + xl * yh  # exact in FP64 for these short significands
    return np.abs(p - x * y) / np.abs(x * y)


def test_bf16x3_products_are_within_3_times_2_to_the_minus_16():
    e = _product_rel_err(_bf16_rne)
    assert e.max() <= 3 * 2.0**-16, e.max()
    assert e.max() >= 3 * 2.0**-19  # the bound is tight: a 16-bit significand pair


def test_3xtf32_products_are_within_2_to_the_minus_20():
    e = _product_rel_err(_tf32_rna)
    assert e.max() <= 3 * 2.0**-22 + 2.0**-23, e.max()
    assert e.max() >= 2.0**-23  # FP32-class, not better


def test_a_dropped_cross_term_is_caught():
    """The mistake the bound must catch: hi*hi + hi*lo alone (lo*hi dropped)."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal(10000)
    y = rng.standard_normal(10000)
    xh, xl = _split(x, _tf32_rna)
    yh, yl = _split(y, _tf32_rna)
    e = np.abs(xh * yh + xh * yl - x * y) / np.abs(x * y)
    assert e.max() > 3 * 2.0**-22 + 2.0**-23


def test_rounding_helpers_match_their_definitions():
    # BF16: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1); 1 + 3 * 2^-8 -> 1 + 2^-6
    v = np.array([1 + 2.0**-8, 1 + 3 * 2.0**-8, -(1 + 2.0**-8)], dtype=np.float32)
    assert np.array_equal(_bf16_rne(v), np.array([1.0, 1 + 2.0**-6, -1.0], dtype=np.float32))
    # TF32: 1 + 2^-11 is a tie between 1 and 1 + 2^-10 -> away (1 + 2^-10)
    w = np.array([1 + 2.0**-11, -(1 + 2.0**-11), 1 + 2.0**-12], dtype=np.float32)
    assert np.array_equal(_tf32_rna(w), np.array([1 + 2.0**-10, -(1 + 2.0**-10), 1.0], dtype=np.float32))
