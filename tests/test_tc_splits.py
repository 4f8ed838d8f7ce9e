"""CPU checks of the precision of the BF16 splits behind the two tensor-core contractions. Each
kernel's split is restated in numpy and compared with exact products: a product of two FP32
numbers, or of two BF16 parts, is exact in FP64.

A round-to-nearest-even conversion to BF16 keeps 8 significant bits, so it moves a value by at
most 2^-8 of itself.

* Forward M (three parts, as in m_operand_kernel): h = bf16(x), m = bf16(x - h) and
  l = bf16(x - h - m), with both differences formed in FP32.
  * Both differences are exact.
  * The last difference has at most 8 significant bits, so x = h + m + l exactly for every
    normal FP32 x above BF16's subnormal range.
  * The six products kept (mm', hl', lh', hm', mh', hh') miss only ml' + lm' + ll', which is at
    most (2 * 2^-24 + 2^-32) |x y|, about 2^-23 of the product.
* Backward dk/dM contraction (two parts, as in split_bf16): hi = bf16(x), lo = bf16(x - hi).
  * The three products kept (hi hi' + hi lo' + lo hi') differ from x y by the rounding of lo and
    lo' (at most 2^-16 of |x y| each) and the dropped lo lo' (about 2^-16).
  * Together that is about 3 * 2^-16 of the product: 4.6e-5 per product.
"""
import numpy as np


def bf16(x):
    """FP32 -> BF16 (returned as FP32 values), round to nearest even: the conversion the kernels
    use.  Finite inputs only."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split3(x):
    h = bf16(x)
    r1 = (x - h).astype(np.float32)
    m = bf16(r1)
    l = bf16((r1 - m).astype(np.float32))
    return h, m, l


def split2(x):
    hi = bf16(x)
    lo = bf16((x - hi).astype(np.float32))
    return hi, lo


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def _samples(seed, n=400_000):
    """Random FP32 values of magnitudes 2^-60 .. 2^60 and both signs, plus edge cases: powers of
    two, values just below them (h rounds up to the next power), halfway cases of the first
    rounding, and all-ones significands."""
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(n) * np.exp2(rng.integers(-60, 60, n))).astype(np.float32)
    e = np.arange(-60, 61, dtype=np.float64)
    p2 = np.exp2(e)
    edge = [p2, np.nextafter(p2.astype(np.float32), np.float32(0)).astype(np.float64),
            p2 * (1 + 2.0 ** -8), p2 * (1 + 3 * 2.0 ** -8), p2 * (2 - 2.0 ** -23),
            p2 * (1 + 2.0 ** -8 + 2.0 ** -16), p2 * (1 + 2.0 ** -9)]
    edge = np.concatenate(edge).astype(np.float32)
    return np.concatenate([x, edge, -edge])


def test_bf16_rounding_is_to_nearest_even():
    # exact BF16 values stay; halfway cases go to the even significand; others to the nearer one
    assert bf16(np.float32(1.0)) == 1.0
    assert bf16(np.float32(1 + 2.0 ** -8)) == 1.0                       # tie, down to even
    assert bf16(np.float32(1 + 3 * 2.0 ** -8)) == np.float32(1 + 2.0 ** -6)  # tie, up to even
    assert bf16(np.float32(1 + 2.0 ** -8 + 2.0 ** -20)) == np.float32(1 + 2.0 ** -7)
    assert bf16(np.float32(-(1 + 2.0 ** -8 + 2.0 ** -20))) == np.float32(-(1 + 2.0 ** -7))
    x = _samples(1)
    rel = np.abs(_f64(bf16(x)) - _f64(x)) / np.abs(_f64(x))
    assert rel.max() <= 2.0 ** -8


def test_three_part_split_is_exact():
    x = _samples(2)
    h, m, l = split3(x)
    r1 = (x - h).astype(np.float32)
    assert np.array_equal(_f64(r1), _f64(x) - _f64(h))                      # x - h exact in FP32
    assert np.array_equal(_f64((r1 - m).astype(np.float32)), _f64(r1) - _f64(m))
    assert np.array_equal(_f64(h) + _f64(m) + _f64(l), _f64(x))             # nothing left over
    assert np.all(np.abs(_f64(m)) <= 2.0 ** -8 * np.abs(_f64(x)))
    assert np.all(np.abs(_f64(l)) <= 2.0 ** -16 * np.abs(_f64(x)))


def test_six_of_nine_products_are_within_two_to_the_minus_23():
    x, y = _samples(3), _samples(4)
    hx, mx, lx = (_f64(v) for v in split3(x))
    hy, my, ly = (_f64(v) for v in split3(y))
    exact = _f64(x) * _f64(y)
    six = mx * my + hx * ly + lx * hy + hx * my + mx * hy + hx * hy
    rel = np.abs(six - exact) / np.abs(exact)
    assert rel.max() <= (2 * 2.0 ** -24 + 2.0 ** -32)
    # the dropped terms are exactly ml' + lm' + ll'
    assert np.allclose(exact - six, mx * ly + lx * my + lx * ly, rtol=0, atol=0)


def test_two_part_products_are_within_three_times_two_to_the_minus_16():
    x, y = _samples(5), _samples(6)
    hx, lx = (_f64(v) for v in split2(x))
    hy, ly = (_f64(v) for v in split2(y))
    exact = _f64(x) * _f64(y)
    three = hx * hy + hx * ly + lx * hy
    rel = np.abs(three - exact) / np.abs(exact)
    bound = 2.0 ** -16 * (2 + 2.0 ** -16 + (1 + 2.0 ** -8) ** 2)
    assert rel.max() <= bound
    # and the bound is of the right order: random pairs come within a factor 2 of it
    assert rel.max() > bound / 2
