"""The three-term TF32 split of the FP32 tensor-core GEMMs (the mixed path's interior
elimination), emulated in NumPy on the CPU: x = x_hi + x_lo with x_hi the TF32 value nearest to
x (10 stored mantissa bits, ties away from zero, the rounding of the kernel's bit operation) and
x_lo = tf32(x - x_hi); a b is taken as a_hi b_hi + a_hi b_lo + a_lo b_hi.  Checked: the split
is exact up to 2^-22 |x|, every product keeps FP32-level accuracy (below 2^-20 |a b|, where one
TF32 product is only good to ~2^-11), and a 128-term dot product stays within 2^-20 sum |a_k b_k|
before the accumulator's own rounding."""
import numpy as np


def tf32(x):
    """Nearest TF32 value of float32 x, ties away from zero: add half a unit of the 13 dropped
    mantissa bits to the magnitude's bit pattern, then clear them."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def split(x):
    x = np.asarray(x, dtype=np.float32)
    hi = tf32(x)
    lo = tf32(x - hi)          # x - hi is exact in FP32
    return hi, lo


def _samples(rng, n):
    return (rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, size=n))).astype(np.float32)


def test_tf32_rounding():
    # 1 + 2^-11 is a tie between 1 and 1 + 2^-10: away from zero; just below it rounds down
    one = np.float32(1.0)
    assert tf32(np.float32(1 + 2.0 ** -11)) == np.float32(1 + 2.0 ** -10)
    assert tf32(np.nextafter(np.float32(1 + 2.0 ** -11), one)) == one
    assert tf32(np.float32(-(1 + 2.0 ** -11))) == np.float32(-(1 + 2.0 ** -10))
    rng = np.random.default_rng(3)
    x = _samples(rng, 10000)
    t = tf32(x)
    assert np.all(t.view(np.uint32) & np.uint32(0x1FFF) == 0)            # 10 mantissa bits left
    assert np.all(np.abs(t.astype(np.float64) - x) <= 2.0 ** -11 * np.abs(x.astype(np.float64)))


def test_split_and_products_keep_fp32_accuracy():
    rng = np.random.default_rng(4)
    a, b = _samples(rng, 20000), _samples(rng, 20000)
    ah, al = split(a)
    bh, bl = split(b)
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    assert np.all(np.abs(ah.astype(np.float64) + al - a64) <= 2.0 ** -22 * np.abs(a64))
    three = ah.astype(np.float64) * bh + ah.astype(np.float64) * bl + al.astype(np.float64) * bh
    one = ah.astype(np.float64) * bh
    exact = a64 * b64
    rel3 = np.abs(three - exact) / np.abs(exact)
    rel1 = np.abs(one - exact) / np.abs(exact)
    assert rel3.max() < 2.0 ** -20, rel3.max()
    assert rel1.max() > 2.0 ** -12          # one TF32 product alone is far from FP32 accuracy


def test_dot_products_of_128_terms():
    rng = np.random.default_rng(5)
    A = np.stack([_samples(rng, 128) for _ in range(64)])
    B = np.stack([_samples(rng, 128) for _ in range(48)])
    Ah, Al = split(A)
    Bh, Bl = split(B)
    f = lambda x: x.astype(np.float64)
    approx = f(Ah) @ f(Bh).T + f(Ah) @ f(Bl).T + f(Al) @ f(Bh).T
    exact = f(A) @ f(B).T
    scale = np.abs(f(A)) @ np.abs(f(B)).T
    assert (np.abs(approx - exact) / scale).max() < 2.0 ** -20
