"""The arithmetic behind the tensor-core contraction of the mixed full Genz
estimate: an FP32 operand x is split into TF32 values hi = round(x) and
lo = round(x - hi) (11 significant bits each, to nearest), and the product
x y is taken as hi_x hi_y + hi_x lo_y + lo_x hi_y.  The dropped lo_x lo_y
and the roundings of lo are each below 2^-22 |x y|, so the three products
reproduce x y to about FP32's own accuracy.  Checked here in numpy on random
FP32 operands, with the rounding written out on the bit patterns."""
import numpy as np


def tf32_round(x):
    """Round float32 values to 11 significant bits (ties away from zero)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return u.view(np.float32)


def _split(x):
    hi = tf32_round(x)
    lo = tf32_round((x - hi).astype(np.float32))
    return hi, lo


def _operands(n, seed):
    rng = np.random.default_rng(seed)
    mag = np.exp2(rng.uniform(-20.0, 20.0, n))
    return (rng.choice([-1.0, 1.0], n) * mag * rng.uniform(1.0, 2.0, n)).astype(np.float32)


def test_tf32_values_have_eleven_significant_bits():
    x = _operands(100_000, 1)
    hi, lo = _split(x)
    for v in (hi, lo):
        bits = v.view(np.uint32)
        assert np.all(bits & 0x1FFF == 0)  # the 13 low mantissa bits are clear
    # hi is the nearest 11-bit value: |x - hi| <= 2^-11 |x|
    assert np.all(np.abs(x.astype(np.float64) - hi) <= 2.0 ** -11 * np.abs(x.astype(np.float64)))


def test_three_products_reproduce_the_fp32_product():
    x, y = _operands(200_000, 2), _operands(200_000, 3)
    hx, lx = _split(x)
    hy, ly = _split(y)
    exact = x.astype(np.float64) * y.astype(np.float64)
    approx = (hx.astype(np.float64) * hy + hx.astype(np.float64) * ly + lx.astype(np.float64) * hy)
    rel = np.abs(approx - exact) / np.abs(exact)
    assert np.max(rel) <= 2.0 ** -20
    # one pass (hi_x hi_y alone) is far coarser: TF32 alone would not do
    one = hx.astype(np.float64) * hy
    assert np.max(np.abs(one - exact) / np.abs(exact)) > 2.0 ** -12


def test_split_is_exact_below_the_second_rounding():
    x = _operands(100_000, 4)
    hi, lo = _split(x)
    resid = x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64)
    assert np.all(np.abs(resid) <= 2.0 ** -22 * np.abs(x.astype(np.float64)))
