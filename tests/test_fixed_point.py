"""The two-word fixed-point split of the gridding kernel, replayed in FP32 on
the host: x = round(v 2^40) (round to nearest even) equals h 2^19 + l, with h
and l read from the bits of two FP32 sums with M = 1.5 2^23.  The products by
2^21 and 2^19 are exact in FP32, so each FMA of the kernel is one FP32 sum
here and the replay is exact."""
import numpy as np

M = np.float32(12582912.0)
MB = 0x4B400000


def split_fixed(v):
    v = np.asarray(v, dtype=np.float32)
    a = v * np.float32(2.0 ** 21) + M          # fmaf(v, 2^21, M): the product is exact
    hf = a - M
    rem = v * np.float32(2.0 ** 21) - hf       # exact: |rem| <= 1/2
    lb = rem * np.float32(2.0 ** 19) + M
    h = a.view(np.int32).astype(np.int64) - MB
    l = lb.view(np.int32).astype(np.int64) - MB
    return h, l


def round_even_2_40(v):
    # v * 2^40 is exact in FP64 for FP32 v; np.rint rounds half to even
    return np.rint(np.asarray(v, dtype=np.float64) * 2.0 ** 40).astype(np.int64)


def test_split_equals_round_to_nearest_even():
    r = np.random.default_rng(40)
    v = np.concatenate([
        r.uniform(-1.999, 1.999, 200000),
        r.uniform(-1e-6, 1e-6, 50000),
        np.ldexp(r.integers(-2 ** 20, 2 ** 20, 50000).astype(np.float64), -41),   # exact halves of 2^-40
        np.ldexp(r.integers(-2 ** 23, 2 ** 23, 50000).astype(np.float64), -22),   # boundaries of h
        [0.0, -0.0, 1.9999999, -1.9999999, 2.0 ** -41, -(2.0 ** -41), 3 * 2.0 ** -41],
    ]).astype(np.float32)
    h, l = split_fixed(v)
    assert np.all(np.abs(l) <= 2 ** 18)
    assert np.all(np.abs(h) <= 2 ** 22)
    assert np.array_equal(h * 2 ** 19 + l, round_even_2_40(v))


def test_word_sums_stay_in_range():
    """8160 terms of the largest |l| stay below 2^31; h sums below 2^31 while
    the item's sum of |v| is below 1023."""
    assert 8160 * 2 ** 18 < 2 ** 31
    assert 2 ** 21 * 1023 + 8160 // 2 + 1 < 2 ** 31
