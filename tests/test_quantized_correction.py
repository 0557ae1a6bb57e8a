"""The arithmetic behind the mixed path's carried residual (the reading of the
correction's precision): once the finest correction v is rounded to a
multiple of q = 2^(E - qb) of a level-wide bound 2^E >= max|v| (qb = 21 for
the 5-point Laplacian, 20 for the 7-point one), the neighbour sum and
L v = sum - 2d c are exact in FP32, so r -= L v can be carried without a
float-float Laplacian; and the float-float update hi + lo <- hi + lo - s2 L v
keeps about 48 bits.  Checked here with IEEE FP32 arithmetic emulated by
numpy (each float32 operation correctly rounded; the fused multiply-add of
the centre term rounded once) against exact FP64 values.  No GPU."""

import math

import numpy as np
import pytest

F32 = np.float32


def magic(bound, qb):
    """M = 1.5 * 2^(E - qb + 23) with E the smallest integer with 2^E >= bound:
    (v + M) - M rounds v to a multiple of 2^(E - qb) for |v| <= 2^E."""
    m, e = math.frexp(bound)  # bound = m 2^e, 0.5 <= m < 1
    E = e - 1 if m == 0.5 else e
    return F32(1.5 * 2.0 ** (E - qb + 23)), E


def quant(v, M):
    return (v.astype(F32) + M) - M  # two correctly rounded float32 operations


def fma32(a, b, c):
    """float32 fused multiply-add: the exact a*b + c (exact in float64 for
    these operands) rounded once to float32."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def _samples(rng, bound, size):
    v = rng.uniform(-bound, bound, size=size)
    v[:8] = [bound, -bound, 0.0, bound * 0.5, -bound * (1 - 2**-24), 2**-140, -(2**-130), bound * 2**-30]
    return v


@pytest.mark.parametrize("bound", [1.0, 0.75, 2.0**-17, 3.1e-9, 1234.5, 2.0**40 * 1.3, 7.0e-30])
def test_rounding_to_the_quantum(bound):
    rng = np.random.default_rng(11)
    for qb in (20, 21):
        M, E = magic(bound, qb)
        q = 2.0 ** (E - qb)
        v = _samples(rng, bound, 4096)
        w = quant(v, M).astype(np.float64)
        assert np.all(np.abs(w - v.astype(F32)) <= q / 2)           # round to nearest multiple
        assert np.all(np.abs(w / q - np.rint(w / q)) == 0.0)        # an exact multiple of q
        assert np.all(np.abs(w) <= 2.0**E)


@pytest.mark.parametrize("dim,qb", [(2, 21), (3, 20)])
@pytest.mark.parametrize("bound", [1.0, 0.75, 2.0**-17, 3.1e-9, 1234.5, 2.0**40 * 1.3])
def test_quantized_laplacian_is_exact_in_fp32(dim, qb, bound):
    rng = np.random.default_rng(12 + dim)
    M, E = magic(bound, qb)
    k = 2 * dim
    nb = [quant(_samples(rng, bound, 20000), M) for _ in range(k)]
    c = quant(_samples(rng, bound, 20000), M)
    # the extreme case: every neighbour at +bound, the centre at -bound
    for a in nb:
        a[8] = quant(np.array([bound]), M)[0]
    c[8] = quant(np.array([-bound]), M)[0]
    if dim == 2:
        s = (nb[0] + nb[1]) + (nb[2] + nb[3])
    else:
        s = ((nb[0] + nb[1]) + (nb[2] + nb[3])) + (nb[4] + nb[5])
    lap = fma32(np.full_like(c, -float(k)), c, s)
    exact = sum(a.astype(np.float64) for a in nb) - k * c.astype(np.float64)
    assert np.array_equal(lap.astype(np.float64), exact)


def test_without_the_rounding_the_fp32_laplacian_is_not_exact():
    """The counter-case: unrounded FP32 values of mixed magnitude lose bits in
    the neighbour sum (so the rounding step is what makes the sum exact)."""
    rng = np.random.default_rng(13)
    nb = [rng.uniform(-1, 1, 20000).astype(F32) for _ in range(4)]
    c = rng.uniform(-1, 1, 20000).astype(F32)
    s = (nb[0] + nb[1]) + (nb[2] + nb[3])
    lap = fma32(np.full_like(c, -4.0), c, s)
    exact = sum(a.astype(np.float64) for a in nb) - 4 * c.astype(np.float64)
    assert not np.array_equal(lap.astype(np.float64), exact)


@pytest.mark.parametrize("dim,qb", [(2, 21), (3, 20)])
def test_headroom_bound(dim, qb):
    """|sum| + 2d |c| <= 4d 2^E stays within 2^24 quanta: the bound that makes
    every intermediate an integer multiple of q representable in FP32."""
    assert 4 * dim * 2.0 ** qb <= 2.0**24


def two_sum32(a, b):
    """Knuth's two-sum in FP32: s = fl(a + b) and the exact error e, a + b = s + e."""
    s = a + b
    bv = s - a
    av = s - bv
    return s, (a - av) + (b - bv)


def ff_sub(hi, lo, lap, s2):
    """(hi + lo) - s2 * lap as a float-float pair; lap exact, s2 a power of two."""
    s, e = two_sum32(hi, -(s2 * lap))
    return two_sum32(s, lo + e)


def test_two_sum_is_exact():
    rng = np.random.default_rng(14)
    a = (rng.uniform(-1, 1, 50000) * 2.0 ** rng.integers(-40, 40, 50000)).astype(F32)
    b = (rng.uniform(-1, 1, 50000) * 2.0 ** rng.integers(-40, 40, 50000)).astype(F32)
    s, e = two_sum32(a, b)
    lhs = a.astype(np.float64) + b.astype(np.float64)  # exact in float64 for these exponent ranges
    assert np.array_equal(s.astype(np.float64) + e.astype(np.float64), lhs)


def test_float_float_update_error():
    """The carried residual's update r <- r - s2 L v keeps about 48 bits: the
    only rounding is that of lo + e, below 2^-47 of |hi| + |s2 L v|."""
    rng = np.random.default_rng(15)
    size = 50000
    hi = (rng.uniform(-1, 1, size) * 2.0 ** rng.integers(-20, 0, size)).astype(F32)
    lo = (hi.astype(np.float64) * rng.uniform(-1, 1, size) * 2.0**-25).astype(F32)
    # a correction of size h^2 |r| (h = 2^-12, the 4095^2 grid) rounded to
    # its quantum; s2 = 1/h^2 = 2^24 is a power of two, so s2 * lap is exact
    b = 2.0**-24
    M, E = magic(b, 21)
    lap = ((quant(rng.uniform(-b, b, size), M) + quant(rng.uniform(-b, b, size), M))
           - F32(2.0) * quant(rng.uniform(-b, b, size), M))
    s2 = F32(2.0**24)
    nh, nl = ff_sub(hi, lo, lap, s2)
    exact = hi.astype(np.float64) + lo.astype(np.float64) - float(s2) * lap.astype(np.float64)
    err = np.abs(nh.astype(np.float64) + nl.astype(np.float64) - exact)
    scale = np.abs(hi.astype(np.float64)) + np.abs(float(s2) * lap.astype(np.float64))
    assert np.all(err <= 2.0**-47 * scale)
    # the pair stays normalised: lo is below half an ulp of hi
    assert np.all(np.abs(nl) <= np.spacing(np.abs(nh)) / 2 + 0.0)
