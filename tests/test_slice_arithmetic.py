"""The floating-point facts the tensor-core operand slicing relies on, checked exhaustively or on
dense samples in NumPy FP32 (the kernels perform the same IEEE-754 operations on the GPU).

* Rounding to the nearest integer, ties to even, by adding and removing 1.5 * 2^23: the same
  value as IEEE rint for FP32 magnitudes below 2^22 (the slices are at most 255.5 in magnitude;
  only the sign of a zero result may differ).
* An integer of magnitude at most 256 is exact in BF16, and its BF16 bits are the upper half of
  its FP32 bits (its low 16 FP32 bits are zero), so a code is a 16-bit shift of the FP32 word.
"""

import numpy as np

ROUND = np.float32(1.5 * 2 ** 23)


def magic_round(t):
    t = np.asarray(t, dtype=np.float32)
    with np.errstate(over="ignore"):
        return (t + ROUND) - ROUND


def test_magic_rounding_equals_rint_over_the_slice_range():
    # FP32 values of the slices' range [-256, 256]: every exponent (subnormals included), each
    # with a dense sample of its mantissas (every 97th bit pattern)
    vals = []
    for e in range(-149, 9):  # subnormals up to 2^8
        lo = np.float32(2.0 ** e)
        bits = np.arange(0, 1 << 23, 97, dtype=np.uint32)  # mantissas, a dense stride
        m = (np.uint32(np.float32(lo).view(np.uint32)) & np.uint32(0x7F800000)) | bits
        vals.append(m.view(np.float32))
    v = np.concatenate(vals)
    v = v[np.isfinite(v) & (np.abs(v) <= 256)]
    for s in (v, -v):
        got = magic_round(s)
        want = np.rint(s)  # IEEE round half to even
        assert np.array_equal(np.abs(got), np.abs(want))
        # equal values; only the sign of zero may differ (a negative value rounding to 0)
        nz = want != 0
        assert np.array_equal(got[nz], want[nz])


def test_magic_rounding_ties_and_limits():
    t = np.array([0.5, 1.5, 2.5, -0.5, -1.5, -2.5, 255.5, -255.5, 127.5, 2 ** 21 + 0.5,
                  2 ** 22 - 0.5, 2 ** 22 - 1.5], dtype=np.float32)
    assert np.array_equal(magic_round(t), np.rint(t))


def test_small_integers_have_bf16_codes_in_their_upper_half():
    c = np.arange(-256, 257, dtype=np.float32)
    bits = c.view(np.uint32)
    assert np.all(bits & np.uint32(0xFFFF) == 0)
    # the BF16 value of the upper half is the integer itself
    back = (bits & np.uint32(0xFFFF0000)).view(np.float32)
    assert np.array_equal(back, c)
    # packing two lanes: (x >> 16) | (y & 0xffff0000), the byte permutation 0x7632
    x, y = bits[:-1], bits[1:]
    packed = (x >> np.uint32(16)) | (y & np.uint32(0xFFFF0000))
    assert np.array_equal((packed & np.uint32(0xFFFF)).astype(np.uint32) << np.uint32(16), x)
    assert np.array_equal(packed & np.uint32(0xFFFF0000), y)
