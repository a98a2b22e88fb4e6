"""Pins of the oracle's radial polynomials against facts fixed outside the oracle.

Each test targets a plausible mistake: a wrong coefficient (orthogonality, the two printed
forms of the radial sum, textbook closed forms), a wrong sign or index (R(1) = 1, the
origin values, R_n^n = rho^n), a wrong derivative (R'(1) closed form, the Jacobi library
routine, symbolic differentiation), or a rounding slip (exact-fraction comparison).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import radial

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DYADIC = [0.0, 0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 1.0]


def all_modes(n_max, m_signed=False):
    for n in range(n_max + 1):
        for m in range(n % 2, n + 1, 2):
            yield n, m


def test_invalid_modes_rejected():
    for n, m in [(-1, 0), (2, 3), (3, 0), (4, 1), (1, -3)]:
        with pytest.raises(ValueError):
            radial.coefficients(n, m)


def test_factorial_form_equals_binomial_form():
    """Sec. 2 prints the radial sum twice: with factorials and with two binomials."""
    for n, m in all_modes(40):
        got = dict(radial.coefficients(n, m))
        for s in range((n - m) // 2 + 1):
            want = (-1) ** s * math.comb(n - s, s) * math.comb(n - 2 * s, (n - m) // 2 - s)
            assert got[n - 2 * s] == want


def test_textbook_closed_forms():
    """Low-order radial polynomials in their classical closed forms (the textbook table the
    paper cites for the radial formula)."""
    closed = {
        (0, 0): lambda r: 1,
        (1, 1): lambda r: r,
        (2, 0): lambda r: 2 * r**2 - 1,
        (2, 2): lambda r: r**2,
        (3, 1): lambda r: 3 * r**3 - 2 * r,
        (3, 3): lambda r: r**3,
        (4, 0): lambda r: 6 * r**4 - 6 * r**2 + 1,
        (4, 2): lambda r: 4 * r**4 - 3 * r**2,
        (5, 1): lambda r: 10 * r**5 - 12 * r**3 + 3 * r,
        (5, 3): lambda r: 5 * r**5 - 4 * r**3,
        (6, 0): lambda r: 20 * r**6 - 30 * r**4 + 12 * r**2 - 1,
        (6, 2): lambda r: 15 * r**6 - 20 * r**4 + 6 * r**2,
    }
    for (n, m), f in closed.items():
        for r in DYADIC + [0.3, 0.91]:
            assert radial.radial_fraction(n, m, 0, r) == f(Fraction(r))


def test_top_mode_and_unit_value():
    """R_n^n = rho^n and R_n^m(1) = 1 (exactly)."""
    for n in range(0, 60):
        for r in [0.3, 0.7, 0.999]:
            assert radial.radial_fraction(n, n, 0, r) == Fraction(r) ** n
    for n, m in all_modes(60):
        assert radial.radial_fraction(n, m, 0, 1.0) == 1


def test_origin_values_golden():
    """Sec. 2: R_n^0(0) = 1 (n = 4k), -1 (n = 4k - 2); every m > 0 vanishes at rho = 0."""
    with open(os.path.join(GOLDEN, "origin_values.txt")) as f:
        rows = [list(map(int, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) > 10
    for n, m, v in rows:
        assert radial.radial(n, m, 0.0) == v
    for n, m in all_modes(30):
        want = 0 if m > 0 or n % 2 else (1 if n % 4 == 0 else -1)
        assert radial.radial_fraction(n, m, 0, 0.0) == want


def test_first_derivative_at_one():
    """R'(1) = (n(n+2) - m^2)/2: from R = (-1)^N rho^m P_N^{(m,0)}(1-2rho^2), the Jacobi
    derivative identity of Sec. 2 and P_N^{(a,b)}(-1) = (-1)^N binom(N+b, N)."""
    for n, m in all_modes(50):
        assert radial.radial_fraction(n, m, 1, 1.0) == Fraction(n * (n + 2) - m * m, 2)


def test_orthogonality_exact():
    """int_0^1 R_n^m R_n'^m rho drho = delta_nn' / (2(n+1)), integrated exactly from the
    integer coefficients."""
    for m in range(0, 9):
        for n1 in range(m, 31, 2):
            c1 = radial.coefficients(n1, m)
            for n2 in range(m, 31, 2):
                c2 = radial.coefficients(n2, m)
                tot = sum(Fraction(a * b, p + q + 2) for p, a in c1 for q, b in c2)
                assert tot == (Fraction(1, 2 * (n1 + 1)) if n1 == n2 else 0)


def test_orthogonality_gauss_legendre_on_values():
    """The evaluated float64 values obey the same orthogonality under Gauss-Legendre
    quadrature in rho (exact for these polynomial degrees)."""
    x, w = np.polynomial.legendre.leggauss(40)
    rho = 0.5 * (x + 1.0)
    w = 0.5 * w
    for m in (0, 1, 3, 8):
        ns = list(range(m, 40, 2))
        vals = np.array(radial.radial_table(ns, [m] * len(ns), rho.tolist(), 0)[0])
        gram = (vals * (w * rho)) @ vals.T
        want = np.diag([1.0 / (2 * (n + 1)) for n in ns])
        assert np.max(np.abs(gram - want)) < 1e-14


def test_jacobi_relation_against_scipy():
    """Sec. 2 Jacobi relation checked against scipy's Jacobi polynomial routine,
    value and first derivative (with the Jacobi derivative identity, k = 1)."""
    sp = pytest.importorskip("scipy.special")
    r = np.linspace(0.0, 1.0, 41)
    x = 1.0 - 2.0 * r**2
    for n, m in all_modes(30):
        N = (n - m) // 2
        want = (-1) ** N * r**m * sp.eval_jacobi(N, m, 0, x)
        got = np.array(radial.radial_table([n], [m], r.tolist(), 1))
        assert np.max(np.abs(got[0][0] - want)) < 1e-12
        dP = 0.0 if N == 0 else 0.5 * (N + m + 1) * sp.eval_jacobi(N - 1, m + 1, 1, x)
        lead = m * r ** (m - 1) if m > 0 else 0.0 * r
        dwant = (-1) ** N * (lead * sp.eval_jacobi(N, m, 0, x) - 4.0 * r ** (m + 1) * dP)
        assert np.max(np.abs(got[1][0] - dwant)) < 1e-10 * max(n, 1) ** 2


def test_derivatives_against_sympy():
    """k = 0..3 against symbolic differentiation of the Jacobi relation (exact rationals)."""
    sympy = pytest.importorskip("sympy")
    rho = sympy.Symbol("rho")
    pts = [Fraction(1, 3), Fraction(5, 8), Fraction(7, 9)]
    for n, m in all_modes(14):
        N = (n - m) // 2
        expr = (-1) ** N * rho**m * sympy.jacobi(N, m, 0, 1 - 2 * rho**2)
        for k in range(4):
            dk = sympy.diff(expr, rho, k)
            coeffs = dict(radial.derivative_coefficients(n, m, k))
            poly = sympy.Poly(sympy.expand(dk), rho)
            for (p,), c in poly.terms():
                assert Fraction(int(c.p), int(c.q)) == coeffs.get(p, 0)
            for q in pts:
                val = sympy.Rational(dk.subs(rho, sympy.Rational(q.numerator, q.denominator)))
                got = sum(c * q**p for p, c in coeffs.items())
                assert Fraction(int(val.p), int(val.q)) == got


def test_kintner_recursion_identity_with_derivatives():
    """Sec. 2 Zernike recursion R_n^m = rho (R_{n-1}^{|m-1|} + R_{n-1}^{m+1}) - R_{n-2}^m (m < n),
    and its k-th derivative rho (A+B)^(k) + k (A+B)^(k-1) - R_{n-2}^m(k), exactly."""
    for r in [0.3, 0.625, 0.95]:
        fr = Fraction(r)
        for n in range(2, 31):
            for m in range(n % 2, n - 1, 2):
                for k in range(4):
                    ab = radial.radial_fraction(n - 1, abs(m - 1), k, r) + radial.radial_fraction(n - 1, m + 1, k, r)
                    rhs = fr * ab - radial.radial_fraction(n - 2, m, k, r)
                    if k:
                        rhs += k * (radial.radial_fraction(n - 1, abs(m - 1), k - 1, r)
                                    + radial.radial_fraction(n - 1, m + 1, k - 1, r))
                    assert radial.radial_fraction(n, m, k, r) == rhs


def test_rounding_is_correct_and_table_layout():
    rs = [0.1, 0.33, 0.5, 0.77, 1.0]
    ns, ms = [4, 7, 100, 4], [2, 3, 0, 2]
    tab = radial.radial_table(ns, ms, rs, 3)
    for k in range(4):
        for j, (n, m) in enumerate(zip(ns, ms)):
            for p, r in enumerate(rs):
                f = radial.radial_fraction(n, m, k, r)
                assert tab[k][j][p] == f.numerator / f.denominator
    assert tab[0][0] == tab[0][3]  # duplicated mode -> identical column


def test_high_order_values_bounded():
    """|R_n^m| <= 1 on [0,1] (a plain property of the radial polynomials), n up to 100."""
    rs = np.linspace(0.0, 1.0, 33).tolist()
    ns, ms = zip(*[(n, m) for n, m in all_modes(100) if n >= 90])
    tab = np.array(radial.radial_table(ns, ms, rs, 0)[0])
    assert np.max(np.abs(tab)) <= 1.0
