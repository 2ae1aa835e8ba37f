"""A CPU model of the integer-field FP64 <-> FP32 conversions the FP32-class
and tensor-core kernels use (f64_to_f32_rn and f32_to_f64 in the kernel
source), checked against the IEEE-754 conversions numpy performs.

The kernels convert on the integer pipe because conversions that involve
FP64 run on the narrow FP64 pipe.  The equivalence argument is pinned here:
* FP32 -> FP64 is exact for every normal FP32 value and zero;
* FP64 -> FP32 rounds to nearest, like the IEEE conversion everywhere except
  at exact ties (which go away from zero), carries a full mantissa into the
  exponent, flushes magnitudes below 2^-126 to a signed zero and sends
  magnitudes beyond the FP32 range to infinity.
The model restates the kernels' bit operations one for one."""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1


def _f64_to_f32_model(x: np.ndarray) -> np.ndarray:
    b = x.astype(np.float64).view(np.uint64).astype(object)
    out = np.empty(x.shape, dtype=np.uint32)
    for i, bi in enumerate(b.ravel()):
        sign = (bi >> 32) & 0x80000000
        mag = bi & 0x7FFFFFFFFFFFFFFF
        em = ((mag + (1 << 28)) >> 29) - ((1023 - 127) << 23)
        bits = (sign | em) & 0xFFFFFFFF if em >= 0 else sign
        if em < (1 << 23):
            bits = sign
        if em >= (255 << 23):
            bits = sign | 0x7F800000
        out.ravel()[i] = bits
    return out.view(np.float32)


def _f32_to_f64_model(f: np.ndarray) -> np.ndarray:
    b = f.astype(np.float32).view(np.uint32).astype(object)
    out = np.empty(f.shape, dtype=np.uint64)
    for i, bi in enumerate(b.ravel()):
        sign = bi & 0x80000000
        e = (bi >> 23) & 0xFF
        mant = bi & 0x7FFFFF
        hi = sign | (((e + (1023 - 127)) << 20) & 0xFFFFFFFF) | (mant >> 3)
        lo = (mant << 29) & 0xFFFFFFFF
        if e == 0:
            hi, lo = sign, 0
        out.ravel()[i] = ((hi << 32) | lo) & M64
    return out.view(np.float64)


def test_fp32_to_fp64_is_exact():
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2 ** 32, size=4000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    e = (bits >> 23) & 0xFF
    f = f[(e > 0) & (e < 255)]  # normal values (the kernels never see others)
    edge = np.array([0.0, -0.0, 1.0, -1.0, np.finfo(np.float32).tiny, np.finfo(np.float32).max,
                     -np.finfo(np.float32).max, np.nextafter(np.float32(1), np.float32(2))], dtype=np.float32)
    f = np.concatenate([f, edge])
    got = _f32_to_f64_model(f)
    assert np.array_equal(got.view(np.uint64), f.astype(np.float64).view(np.uint64))
    # subnormal inputs (never produced by the flushing conversion) map to a signed zero
    sub = np.array([1e-40, -1e-40], dtype=np.float32)
    assert np.array_equal(_f32_to_f64_model(sub), np.array([0.0, -0.0])) and np.signbit(_f32_to_f64_model(sub)[1])


def test_fp64_to_fp32_rounds_to_nearest():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(3000) * np.exp(rng.uniform(-80, 80, size=3000))
    got = _f64_to_f32_model(x)
    ref = x.astype(np.float32)  # IEEE round to nearest, ties to even
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_fp64_to_fp32_edges():
    f32 = np.float32
    one = 1.0
    ulp = 2.0 ** -23
    # exact ties go away from zero (the IEEE conversion takes the even one)
    ties = np.array([one + 0.5 * ulp, -(one + 0.5 * ulp), one + 2.5 * ulp])
    got = _f64_to_f32_model(ties).astype(np.float64)
    assert got.tolist() == [one + ulp, -(one + ulp), one + 3 * ulp]
    # a full mantissa rounds up into the next binade
    x = np.array([2.0 - 0.25 * ulp, np.nextafter(2.0, 0.0)])
    assert _f64_to_f32_model(x).tolist() == [2.0, 2.0]
    # below 2^-126 (the smallest normal FP32): signed zero; beyond the range: infinity
    tiny = float(np.finfo(f32).tiny)
    small = np.array([0.75 * tiny, -0.75 * tiny, 1e-300, 0.0, -0.0])
    got = _f64_to_f32_model(small)
    assert np.all(got == 0.0) and np.array_equal(np.signbit(got), np.signbit(small))
    assert _f64_to_f32_model(np.array([tiny]))[0] == f32(tiny)
    fmax = float(np.finfo(f32).max)
    # from max + half an ulp (2^103) on, the nearest is beyond the range
    big = np.array([1e39, -1e300, fmax + 2.0 ** 103, fmax + 2.0 ** 102])
    assert _f64_to_f32_model(big).tolist() == [np.inf, -np.inf, np.inf, fmax]
    with np.errstate(over="ignore"):
        assert big[2:].astype(f32).tolist() == [np.inf, fmax]  # the IEEE conversion agrees
    assert _f64_to_f32_model(np.array([float(np.finfo(f32).max)]))[0] == np.finfo(f32).max
    # and the round trip of any FP32 value is the identity
    rng = np.random.default_rng(3)
    f = (rng.standard_normal(2000) * np.exp(rng.uniform(-60, 60, size=2000))).astype(f32)
    assert np.array_equal(_f64_to_f32_model(_f32_to_f64_model(f)).view(np.uint32), f.view(np.uint32))
