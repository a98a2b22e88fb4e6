"""cos(t) and sin(t) for an exact rational t, in big-integer fixed point.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The angular factor of Z_n^m (paper Sec. 2, definition of Z: cos(m theta) for m >= 0,
sin(|m| theta) for m < 0) is evaluated here at theta's exact float64 value, to about
WORK_BITS - 16 bits, far above the 54 decimal digits (about 180 bits) that the paper's
precision appendix finds sufficient for the radial sum.  No third-party arbitrary-precision
package is needed, so the oracle runs wherever Python runs.

Method (textbook, written out plainly):
  * pi from Machin's formula pi = 16 atan(1/5) - 4 atan(1/239), each arctangent by its
    alternating Taylor series, in fixed point with guard bits;
  * argument reduction t = q * (pi/2) + u with |u| <= pi/4 (q the nearest integer);
  * Taylor series of cos(u) and sin(u) until the terms vanish;
  * quadrant rotation by q mod 4.
Every fixed-point value is an integer X standing for X / 2^WORK_BITS.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

WORK_BITS = 320
GUARD_BITS = 64


def _atan_inv(x: int, bits: int) -> int:
    """atan(1/x) * 2^bits by the series sum_i (-1)^i / ((2i+1) x^(2i+1)), truncated."""
    power = (1 << bits) // x
    total = power
    x2 = x * x
    i = 1
    while power:
        power //= x2
        term = power // (2 * i + 1)
        total = total - term if i % 2 else total + term
        i += 1
    return total


@lru_cache(maxsize=None)
def pi_fixed(bits: int = WORK_BITS) -> int:
    """pi * 2^bits (error below one unit in the last place)."""
    b = bits + GUARD_BITS
    pi_big = 16 * _atan_inv(5, b) - 4 * _atan_inv(239, b)
    return pi_big >> GUARD_BITS


def _to_fixed(t: Fraction, bits: int) -> int:
    return (t.numerator << bits) // t.denominator


def cos_sin_fixed(t: Fraction, bits: int = WORK_BITS) -> tuple[int, int]:
    """(cos t, sin t) * 2^bits as integers for an exact rational t."""
    b = bits + GUARD_BITS
    one = 1 << b
    T = _to_fixed(Fraction(t), b)
    half_pi = pi_fixed(b) >> 1
    q = (T + (half_pi >> 1)) // half_pi
    u = T - q * half_pi
    u2 = (u * u) >> b
    # cos(u) = sum (-1)^i u^(2i) / (2i)!,  sin(u) = sum (-1)^i u^(2i+1) / (2i+1)!
    c_term, c_sum = one, one
    s_term, s_sum = u, u
    i = 1
    while c_term or s_term:
        c_term = -((c_term * u2) >> b) // ((2 * i - 1) * (2 * i))
        s_term = -((s_term * u2) >> b) // ((2 * i) * (2 * i + 1))
        c_sum += c_term
        s_sum += s_term
        i += 1
        if i > 10_000:  # |u| <= pi/4 converges in well under 100 terms
            raise RuntimeError("trig series did not converge")
    quadrant = q % 4
    if quadrant == 0:
        c, s = c_sum, s_sum
    elif quadrant == 1:
        c, s = -s_sum, c_sum
    elif quadrant == 2:
        c, s = -c_sum, -s_sum
    else:
        c, s = s_sum, -c_sum
    return c >> GUARD_BITS, s >> GUARD_BITS


@lru_cache(maxsize=1 << 16)
def cos_sin_multiple(m: int, theta: float, bits: int = WORK_BITS) -> tuple[int, int]:
    """(cos(m theta), sin(m theta)) * 2^bits for an integer m and theta's exact float64 value."""
    return cos_sin_fixed(Fraction(m) * Fraction(float(theta)), bits)


def cos_multiple(m: int, theta: float) -> float:
    """cos(m theta) rounded to float64."""
    c, _ = cos_sin_multiple(m, theta)
    return c / (1 << WORK_BITS)


def sin_multiple(m: int, theta: float) -> float:
    """sin(m theta) rounded to float64."""
    _, s = cos_sin_multiple(m, theta)
    return s / (1 << WORK_BITS)
