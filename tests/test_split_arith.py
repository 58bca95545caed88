"""Host checks of the FP32 identities the split-BF16 GEMM's epilogue relies on
(no GPU): FP32 arithmetic is emulated with numpy float32, whose operations
round to nearest even like the kernel's.

* Magic-number rounding: for |y| <= 2^22, float32(y + 1.5 * 2^23) has the
  integer round(y) (ties to even) in its low mantissa bits.
* The final drain's round(acc3 * 2^24) for |acc3| < 64: h = round(acc3 * 2^16)
  by the magic number, the remainder acc3 - h 2^-16 exact in FP32, and
  round(acc3 * 2^24) = 2^8 h + round(remainder * 2^24)."""
import numpy as np

F = np.float32
M0 = F(12582912.0)  # 1.5 * 2^23
B0 = int(np.array(M0, dtype=np.float32).view(np.int32))


def magic_round(y):
    """round(y) via the magic number (y float32, |y| <= 2^22).  y + M0 is one
    float32 addition, as the kernel's fma(x, 2^k, M0) is when x 2^k is exact."""
    with np.errstate(all="ignore"):
        return (y + M0).view(np.int32).astype(np.int64) - B0


def acc3_scaled(x):
    """The epilogue's round(x * 2^24) with FP32 operations only."""
    r = x * F(65536.0) + M0
    rem = x - (r - M0) * F(1.0 / 65536.0)
    h = r.view(np.int32).astype(np.int64) - B0
    return (h << 8) + magic_round(rem * F(16777216.0))


def test_magic_round_ties_to_even():
    k = np.arange(-2 ** 12, 2 ** 12, dtype=np.int64)
    for frac in (0.0, 0.25, 0.5, 0.75):
        y = (k + frac).astype(np.float32)
        assert np.array_equal(magic_round(y), np.rint(y.astype(np.float64)).astype(np.int64))
    big = np.array([2.0 ** 22, -2.0 ** 22, 2.0 ** 22 - 0.5, -(2.0 ** 22) + 0.5], dtype=np.float32)
    assert np.array_equal(magic_round(big), np.rint(big.astype(np.float64)).astype(np.int64))


def test_acc3_rounding_matches_float64():
    rng = np.random.default_rng(11)
    xs = [(rng.standard_normal(4000) * 2.0 ** e).astype(np.float32) for e in range(-40, 6)]
    k = rng.integers(-2 ** 29, 2 ** 29, 20000)
    xs.append(((k + 0.5) * 2.0 ** -24).astype(np.float32))   # exact ties at 2^-24
    xs.append((k * 2.0 ** -24).astype(np.float32))
    xs.append(np.array([0.0, -0.0, 63.99, -63.99, 2.0 ** -17, -(2.0 ** -17), 1.5 * 2.0 ** -16,
                        3 * 2.0 ** -25], dtype=np.float32))
    x = np.concatenate(xs)
    x = x[np.abs(x) < 64]
    want = np.rint(x.astype(np.float64) * 2.0 ** 24).astype(np.int64)
    assert np.array_equal(acc3_scaled(x), want)


def test_drain_bound_fits_the_magic_window():
    """A drain carries at most 3 x 64, 2 x 128 or 1 x 256 slice products of
    |a_i b_j| <= 2^14 (diagonals 2, 1, 0), so the FP32 sum is an integer
    within the magic-number window 2^22."""
    assert max(3 * 64, 2 * 128, 1 * 256) * 2 ** 14 <= 2 ** 22
