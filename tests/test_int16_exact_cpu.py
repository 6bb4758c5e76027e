"""The exact INT16 conversions the 16-bit kernels rely on, checked on the CPU
for every 16-bit value.

The INT16 form stores q in [-32767, 32767] in offset binary, u = q + 32768.
- Tensor-core kernels split u into two FP16 numbers, both exact: from the
  high byte b1 the number with bits 0x6400 | b1 (= 1024 + b1), minus 1152,
  times 256; from the low byte b0 the number 0x6400 | b0, minus 1024.  Their
  sum is q.  The halves of a 32-bit word (two values) are formed by byte
  permutes with selectors 0x4240 (bytes b0, 0x64, b2, 0x64) and 0x4341
  (bytes b1, 0x64, b3, 0x64).
- The CUDA-core near field places u under the exponent of 2^23 (bits
  0x4B000000 | u, the float 2^23 + u) and subtracts 2^23 + 2^15.
Each step must be exact in the arithmetic the kernels use (FP16 subtraction
and multiplication, FP32 subtraction); numpy's float16 and float32 round the
same way (round to nearest even), so an exact result here is exact there.
"""
import numpy as np

U = np.arange(65536, dtype=np.uint32)  # every offset-binary value
Q = U.astype(np.int64) - 32768


def byte_perm(x, y, s):
    """The byte permute of two 32-bit words (selector nibbles 0-3 pick bytes of
    x, 4-7 bytes of y), as the kernels use it."""
    b = [(x >> (8 * i)) & 0xFF for i in range(4)] + [(y >> (8 * i)) & 0xFF for i in range(4)]
    r = np.zeros_like(x)
    for n in range(4):
        r |= b[(s >> (4 * n)) & 7] << (8 * n)
    return r


def test_byte_permute_selectors_form_the_fp16_patterns():
    rng = np.random.default_rng(3)
    w = rng.integers(0, 2 ** 32, 100000, dtype=np.uint64).astype(np.uint32)
    fill = np.full_like(w, 0x64646464)
    np.testing.assert_array_equal(byte_perm(w, fill, 0x4240), (w & 0x00FF00FF) | 0x64006400)
    np.testing.assert_array_equal(byte_perm(w, fill, 0x4341), ((w >> 8) & 0x00FF00FF) | 0x64006400)


def test_fp16_split_of_every_int16_value_is_exact():
    lo_bits = ((U & 0xFF) | 0x6400).astype(np.uint16)
    hi_bits = ((U >> 8) | 0x6400).astype(np.uint16)
    lo16 = lo_bits.view(np.float16)
    hi16 = hi_bits.view(np.float16)
    np.testing.assert_array_equal(lo16.astype(np.int64), 1024 + (U & 0xFF))
    np.testing.assert_array_equal(hi16.astype(np.int64), 1024 + (U >> 8))
    lo = lo16 - np.float16(1024.0)
    hi = (hi16 - np.float16(1152.0)) * np.float16(256.0)
    assert lo.dtype == np.float16 and hi.dtype == np.float16
    np.testing.assert_array_equal(lo.astype(np.int64), U & 0xFF)
    np.testing.assert_array_equal(hi.astype(np.int64), 256 * ((U >> 8).astype(np.int64) - 128))
    np.testing.assert_array_equal(hi.astype(np.int64) + lo.astype(np.int64), Q)
    # both halves carry at most 8 significant bits: any FP16 operand of an
    # MMA product with them keeps the product exact in the FP32 accumulator
    assert np.abs(lo.astype(np.float64)).max() <= 255
    assert np.abs(hi.astype(np.float64)).max() <= 32768


def test_float32_exponent_trick_of_every_int16_value_is_exact():
    f = (U | 0x4B000000).view(np.float32)
    np.testing.assert_array_equal(f.astype(np.float64), 8388608.0 + U)
    q = f - np.float32(8421376.0)
    assert q.dtype == np.float32
    np.testing.assert_array_equal(q.astype(np.int64), Q)
