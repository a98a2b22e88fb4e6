"""Exact radial Zernike polynomials R_n^{|m|}(rho) and their rho-derivatives.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definition followed: paper Sec. 2, the explicit radial sum
    R_n^{|m|}(rho) = sum_{s=0}^{(n-|m|)/2} (-1)^s (n-s)! / ( s! ((n+|m|)/2 - s)! ((n-|m|)/2 - s)! ) rho^{n-2s}
The coefficients are integers (the paper's remark after the binomial form), so they are
formed with exact Python integers and exact integer division.  Derivatives differentiate
each monomial exactly: d^k/drho^k rho^p = p (p-1) ... (p-k+1) rho^{p-k} (zero when p < k).
A float64 input r is an exact dyadic rational, so each value is an exact rational that is
rounded once to float64 (Python's int / int true division rounds correctly).

Derivative variable: rho (the radial coordinate), not the Jacobi argument x = 1 - 2 rho^2.
Mode rule (Sec. 2): n >= 0, |m| <= n, n - |m| even; anything else raises ValueError.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import factorial


def check_mode(n: int, m: int) -> None:
    """Raise ValueError unless n >= 0, |m| <= n and n - |m| is even (Sec. 2)."""
    if n < 0 or abs(m) > n or (n - abs(m)) % 2 != 0:
        raise ValueError(f"invalid Zernike mode (n={n}, m={m})")


@lru_cache(maxsize=None)
def coefficients(n: int, m: int) -> tuple[tuple[int, int], ...]:
    """((power, integer coefficient), ...) of R_n^{|m|}, one entry per s = 0..(n-|m|)/2,
    from the factorial form of the radial sum (Sec. 2)."""
    check_mode(n, m)
    m = abs(m)
    out = []
    for s in range((n - m) // 2 + 1):
        num = factorial(n - s)
        den = factorial(s) * factorial((n + m) // 2 - s) * factorial((n - m) // 2 - s)
        q, rem = divmod(num, den)
        assert rem == 0, "radial coefficients are integers"
        out.append((n - 2 * s, -q if s % 2 else q))
    return tuple(out)


@lru_cache(maxsize=None)
def derivative_coefficients(n: int, m: int, k: int) -> tuple[tuple[int, int], ...]:
    """((power, integer coefficient), ...) of d^k/drho^k R_n^{|m|} (monomials with p < k vanish)."""
    if k < 0:
        raise ValueError("derivative order must be >= 0")
    out = []
    for p, c in coefficients(n, m):
        if p < k:
            continue
        ff = 1
        for i in range(k):
            ff *= p - i
        out.append((p - k, c * ff))
    return tuple(out)


def _dyadic(x: float) -> tuple[int, int]:
    """x = a / 2^e exactly (e >= 0)."""
    a, d = float(x).as_integer_ratio()
    e = d.bit_length() - 1
    assert d == 1 << e
    return a, e


def radial_fraction(n: int, m: int, k: int, r: float) -> Fraction:
    """Exact rational value of d^k/drho^k R_n^{|m|} at the float64 r."""
    a, e = _dyadic(r)
    coeffs = derivative_coefficients(n, m, k)
    if not coeffs:
        return Fraction(0)
    pmax = max(p for p, _ in coeffs)
    num = 0
    for p, c in coeffs:
        num += c * a ** p * (1 << (e * (pmax - p)))
    return Fraction(num, 1 << (e * pmax))


class PointPowers:
    """Powers of one float64 point r = a / 2^e, all over the common denominator 2^(e*pmax):
    r^p = pw[p] / 2^(e*pmax).  Lets many modes share the big-integer powers."""

    def __init__(self, r: float, pmax: int):
        a, e = _dyadic(r)
        self.pmax = pmax
        self.shift = e * pmax
        pw = [0] * (pmax + 1)
        ap = 1
        for p in range(pmax + 1):
            pw[p] = ap << (e * (pmax - p))
            ap *= a
        self.pw = pw

    def value(self, coeffs) -> float:
        num = 0
        pw = self.pw
        for p, c in coeffs:
            num += c * pw[p]
        return num / (1 << self.shift)  # int / int: correctly rounded

    def fraction(self, coeffs) -> Fraction:
        num = 0
        for p, c in coeffs:
            num += c * self.pw[p]
        return Fraction(num, 1 << self.shift)


def radial(n: int, m: int, r: float, k: int = 0) -> float:
    """d^k/drho^k R_n^{|m|}(r) rounded once to float64."""
    f = radial_fraction(n, m, k, r)
    return f.numerator / f.denominator


def radial_table(ns, ms, rs, max_deriv: int = 0):
    """out[k][j][p] = d^k/drho^k R_{n_j}^{|m_j|}(r_p) for k = 0..max_deriv, as nested lists of
    float64 (column order = the caller's mode order; duplicates allowed)."""
    ns = [int(v) for v in ns]
    ms = [int(v) for v in ms]
    for n, m in zip(ns, ms):
        check_mode(n, m)
    pmax = max(ns) if ns else 0
    out = [[[0.0] * len(rs) for _ in ns] for _ in range(max_deriv + 1)]
    for p, r in enumerate(rs):
        pp = PointPowers(float(r), pmax)
        for j, (n, m) in enumerate(zip(ns, ms)):
            for k in range(max_deriv + 1):
                out[k][j][p] = pp.value(derivative_coefficients(n, m, k))
    return out
