"""The variability kernel rounds each direction component x to the fixed-point
integer llrint(x * 2^40) in fp32 arithmetic, as hi * 2^22 + lo with
hi = rint(x * 2^18) and lo = rint((x * 2^18 - hi) * 2^22), each rint done by
adding 1.5 * 2^23.  This checks that identity (the same float32 steps in
numpy) against the exact FP64 product on every exponent, on exact ties and on
boundary values.  It imports neither the oracle nor the library."""
import numpy as np

C = np.float32(12582912.0)           # 1.5 * 2^23


def split(x):
    x = np.asarray(x, np.float32)
    t = (x * np.float32(262144.0)).astype(np.float32)                 # x * 2^18 (exact)
    a = (t + C).astype(np.float32)                                     # C + rint(t)
    hi = a.view(np.int32).astype(np.int64) - C.view(np.int32).astype(np.int64)
    r = (t - (a - C).astype(np.float32)).astype(np.float32)            # t - rint(t) (exact)
    b = ((r * np.float32(4194304.0)).astype(np.float32) + C).astype(np.float32)
    lo = b.view(np.int32).astype(np.int64) - C.view(np.int32).astype(np.int64)
    return (hi << 22) + lo


def exact(x):
    return np.rint(np.asarray(x, np.float32).astype(np.float64) * 2.0 ** 40).astype(np.int64)


def test_random_bit_patterns():
    rng = np.random.default_rng(7)
    x = rng.integers(0, 2 ** 32, 4_000_000, dtype=np.int64).astype(np.uint32).view(np.float32)
    x = x[np.isfinite(x) & (np.abs(x) < 8.0)]
    assert len(x) > 1_000_000
    assert np.array_equal(split(x), exact(x))


def test_exact_ties_round_to_even():
    # x = (2m + 1) * 2^-41: x * 2^40 = m + 1/2 exactly
    rng = np.random.default_rng(8)
    m = rng.integers(0, 2 ** 23, 200_000)
    x = ((2 * m + 1).astype(np.float64) * 2.0 ** -41).astype(np.float32)
    assert np.array_equal(x.astype(np.float64) * 2.0 ** 40 % 1.0, np.full(len(x), 0.5))
    for s in (1.0, -1.0):
        assert np.array_equal(split(s * x), exact(s * x))


def test_boundary_values():
    v = [0.0, -0.0, 1.0, -1.0, 0.5, 2.0 ** -40, 2.0 ** -41, 3 * 2.0 ** -42, 1.5 * 2.0 ** -40, 2.0 ** -126,
         2.0 ** -149, 1 - 2.0 ** -24, -(1 - 2.0 ** -24), 2.0 ** -17, 2.0 ** -18, 2.0 ** -19, 7.999999]
    assert np.array_equal(split(v), exact(v))
