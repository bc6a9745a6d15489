"""CPU check of the integer float -> double conversion used by the FP64 iterate
updates (`f2d_exact` in the CUDA library).

The kernels form the binary64 bits of a binary32 value with integer operations:
high word = sign | ((|bits| >> 3) + (896 << 20)), low word = bits << 29 (the
exponent rebiased from 127 to 1023, the 23 mantissa bits moved up by 29), with
+-0 mapped to a signed zero, and subnormal, inf and NaN inputs left to the
hardware conversion.  The test applies the same integer steps to every binary32
exponent with random mantissas and to the edge values, and compares the bits
with numpy's float32 -> float64 conversion.
"""

import numpy as np


def _f2d_bits(b: np.ndarray) -> np.ndarray:
    b = b.astype(np.uint64)
    a = b & np.uint64(0x7FFFFFFF)
    hi = (b & np.uint64(0x80000000)) | np.where(a == 0, np.uint64(0), (a >> np.uint64(3)) + np.uint64(896 << 20))
    lo = (b << np.uint64(29)) & np.uint64(0xFFFFFFFF)
    return (hi << np.uint64(32)) | lo


def _fast_path(b: np.ndarray) -> np.ndarray:
    a = b & np.uint32(0x7FFFFFFF)
    e = a >> np.uint32(23)
    return ~(((e == 0) & (a != 0)) | (e == 0xFF))


def test_every_normal_exponent_and_zero_match_the_conversion():
    rng = np.random.default_rng(5)
    exps = np.repeat(np.arange(1, 255, dtype=np.uint32), 64)
    mant = rng.integers(0, 1 << 23, exps.size, dtype=np.uint32)
    mant[::64] = 0                      # powers of two
    mant[1::64] = (1 << 23) - 1         # largest mantissa of each binade
    sign = rng.integers(0, 2, exps.size, dtype=np.uint32) << np.uint32(31)
    bits = np.concatenate([sign | (exps << np.uint32(23)) | mant,
                           np.array([0x00000000, 0x80000000], dtype=np.uint32)])
    assert _fast_path(bits).all()
    ref = bits.view(np.float32).astype(np.float64).view(np.uint64)
    np.testing.assert_array_equal(_f2d_bits(bits), ref)


def test_subnormal_inf_and_nan_take_the_hardware_conversion():
    special = np.array([0x00000001, 0x807FFFFF, 0x7F800000, 0xFF800000, 0x7FC00000], dtype=np.uint32)
    assert not _fast_path(special).any()
    # the integer form would be wrong for them (why they are excluded)
    ref = special.view(np.float32).astype(np.float64).view(np.uint64)
    assert (_f2d_bits(special) != ref).all()
