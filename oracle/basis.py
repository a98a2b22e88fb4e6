"""Zernike functions Z_n^m(rho, theta) and their derivatives, rounded once to float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definition followed (paper Sec. 2, definition of Z):
    Z_n^m = R_n^{m}(rho) cos(m theta)        for m >= 0
    Z_n^m = R_n^{|m|}(rho) sin(|m| theta)    for m < 0
with no normalisation factor.  Radial derivatives act on R only:
    d^k/drho^k Z_n^m = R^{(k)}(rho) * (cos or sin)(|m| theta).
The theta derivative is
    d/dtheta Z_n^m = -|m| R sin(|m| theta)  (m >= 0),   +|m| R cos(|m| theta)  (m < 0).
R is the exact rational of oracle.radial; the trig factor is the fixed-point value of
oracle.trig; the product is formed exactly and rounded once.
"""
from __future__ import annotations

from . import radial as _radial
from . import trig as _trig

_ONE_TRIG = 1 << _trig.WORK_BITS


def _angular_fixed(m: int, theta: float) -> int:
    c, s = _trig.cos_sin_multiple(abs(m), theta)
    return c if m >= 0 else s


def _dtheta_fixed(m: int, theta: float) -> int:
    c, s = _trig.cos_sin_multiple(abs(m), theta)
    return -abs(m) * s if m >= 0 else abs(m) * c


def _round_product(num: int, den: int, trig_fixed: int) -> float:
    return (num * trig_fixed) / (den * _ONE_TRIG)


def basis_value(n: int, m: int, r: float, theta: float, k: int = 0) -> float:
    """d^k/drho^k Z_n^m(r, theta), rounded once."""
    f = _radial.radial_fraction(n, m, k, r)
    return _round_product(f.numerator, f.denominator, _angular_fixed(m, theta))


def basis_dtheta(n: int, m: int, r: float, theta: float) -> float:
    """d/dtheta Z_n^m(r, theta), rounded once."""
    f = _radial.radial_fraction(n, m, 0, r)
    return _round_product(f.numerator, f.denominator, _dtheta_fixed(m, theta))


def _dtheta_k_fixed(m: int, theta: float, kt: int) -> int:
    """d^kt/dtheta^kt of cos(|m| theta) (m >= 0) or sin(|m| theta) (m < 0), kt = 0..2, fixed point."""
    c, s = _trig.cos_sin_multiple(abs(m), theta)
    a = abs(m)
    if kt == 0:
        return c if m >= 0 else s
    if kt == 1:
        return -a * s if m >= 0 else a * c
    if kt == 2:
        return -a * a * (c if m >= 0 else s)
    raise ValueError("kt must be 0..2")


def basis_deriv(n: int, m: int, r: float, theta: float, kr: int, kt: int) -> float:
    """d^kr/drho^kr d^kt/dtheta^kt Z_n^m(r, theta) = R^(kr)(r) * (trig)^(kt)(theta), rounded once."""
    f = _radial.radial_fraction(n, m, kr, r)
    return _round_product(f.numerator, f.denominator, _dtheta_k_fixed(m, theta, kt))


def basis_table(ns, ms, rs, thetas, max_deriv: int = 0, with_dtheta: bool = False):
    """Returns (zk, zt): zk[k][j][p] = d^k/drho^k Z_{n_j}^{m_j}(r_p, theta_p), k = 0..max_deriv,
    and zt[j][p] = d/dtheta Z (or None).  Column order = the caller's mode order."""
    ns = [int(v) for v in ns]
    ms = [int(v) for v in ms]
    for n, m in zip(ns, ms):
        _radial.check_mode(n, m)
    pmax = max(ns) if ns else 0
    J, P = len(ns), len(rs)
    zk = [[[0.0] * P for _ in range(J)] for _ in range(max_deriv + 1)]
    zt = [[0.0] * P for _ in range(J)] if with_dtheta else None
    for p in range(P):
        r, th = float(rs[p]), float(thetas[p])
        pp = _radial.PointPowers(r, pmax)
        den = (1 << pp.shift) * _ONE_TRIG
        for j, (n, m) in enumerate(zip(ns, ms)):
            ang = _angular_fixed(m, th)
            for k in range(max_deriv + 1):
                num = 0
                for pw, c in _radial.derivative_coefficients(n, m, k):
                    num += c * pp.pw[pw]
                zk[k][j][p] = (num * ang) / den
            if with_dtheta:
                num = 0
                for pw, c in _radial.coefficients(n, m):
                    num += c * pp.pw[pw]
                zt[j][p] = (num * _dtheta_fixed(m, th)) / den
    return zk, zt
