"""The fixed-point Laplacian of the mixed path's direct residuals, checked on
the CPU against exact rational arithmetic.  Each double of the stencil is
taken as its signed 53-bit significand and exponent, shifted left by g guard
bits and right to the largest exponent of the stencil (bits below that are
truncated toward minus infinity, as an arithmetic shift does), summed
exactly in 64-bit integers, and rounded once to a double scaled by
1/h^2 = 2^lg.  Properties: exact rounding when the exponents are within g of
each other; otherwise an error of at most half an ulp plus the truncation of
the 2d + 1 terms (the centre counted 2d times); no 64-bit overflow."""

import struct
from fractions import Fraction

import numpy as np
import pytest

GUARD = 6


def dec(x):
    b = struct.unpack("<Q", struct.pack("<d", float(x)))[0]
    e = (b >> 52) & 0x7FF
    m = ((b & ((1 << 52) - 1)) | (1 << 52)) if e else 0  # subnormals read as zero
    return (-m if b >> 63 else m), e


def al(a, emax, g=GUARD):
    m, e = a
    k = emax - e
    return 0 if k > 62 else (m << g) >> k


def fixed_lap(center, nbrs, lg, g=GUARD):
    """(sum of neighbours - 2d centre) * 2^lg, the integer way."""
    xs = [dec(center)] + [dec(v) for v in nbrs]
    em = max(e for _, e in xs)
    t = sum(al(a, em, g) for a in xs[1:]) - len(nbrs) * al(xs[0], em, g)
    assert -(1 << 63) <= t < (1 << 63)
    return float(Fraction(t) * Fraction(2) ** (em - 1075 - g + lg)), em  # float(): round to nearest even


def exact_lap(center, nbrs, lg):
    return (sum(Fraction(v) for v in nbrs) - len(nbrs) * Fraction(center)) * Fraction(2) ** lg


def ulp(x):
    return np.spacing(abs(x)) if x != 0 else 0.0


@pytest.mark.parametrize("d", [2, 3])
def test_exactly_rounded_when_exponents_are_close(d):
    rng = np.random.default_rng(21 + d)
    lg = 24  # h = 2^-12
    for _ in range(3000):
        e0 = int(rng.integers(-30, 30))
        vals = [float(rng.uniform(1, 2) * 2.0 ** (e0 - int(rng.integers(0, GUARD + 1))) * rng.choice([-1, 1]))
                for _ in range(2 * d + 1)]
        got, _ = fixed_lap(vals[0], vals[1:], lg)
        assert got == float(exact_lap(vals[0], vals[1:], lg))


@pytest.mark.parametrize("d", [2, 3])
def test_error_bound_for_any_spread(d):
    rng = np.random.default_rng(31 + d)
    lg = 24
    for _ in range(3000):
        vals = [float(rng.uniform(-1, 1) * 2.0 ** int(rng.integers(-70, 5))) for _ in range(2 * d + 1)]
        if rng.random() < 0.1:
            vals[int(rng.integers(0, 2 * d + 1))] = 0.0
        got, em = fixed_lap(vals[0], vals[1:], lg)
        exact = exact_lap(vals[0], vals[1:], lg)
        unit = Fraction(2) ** (em - 1075 - GUARD + lg)
        bound = Fraction(ulp(got)) / 2 + 4 * d * unit  # 2d neighbours + 2d copies of the centre, < 1 unit each
        assert abs(Fraction(got) - exact) <= bound


def test_cancellation_keeps_every_bit():
    """A smooth field: the neighbours nearly cancel the centre, and the
    integer sum keeps all the bits the FP64 partial sums would round away."""
    lg = 24
    c = 0.7390851332151607
    h = 2.0**-12
    nb = [c + 1e-9 * k * h for k in (1, -1, 2, -2)]
    got, _ = fixed_lap(c, nb, lg)
    assert got == float(exact_lap(c, nb, lg))


def test_no_overflow_at_the_extremes():
    """|t| <= (2d + 2d) 2^(53 + g) < 2^63 for g = 6 (second order, 3D); the
    fourth-order stencils use g = 3: weights up to 48 in total, 48 x 2^56 < 2^62."""
    big = float(np.nextafter(2.0, 0.0))  # the largest significand
    got, _ = fixed_lap(-big, [big] * 6, 0)
    assert got == float(exact_lap(-big, [big] * 6, 0))
    assert 12 * 2 ** (53 + GUARD) < 2**63
    assert 48 * 2 ** (53 + 3) < 2**62
