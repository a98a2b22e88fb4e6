"""Pins of the oracle's angular factor, Z_n^m and the series/adjoint definitions."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import basis, radial, series, trig
from paper_2409_19156_gb300 import inputs


def test_pi_matches_known_double_and_mpmath():
    one = 1 << trig.WORK_BITS
    assert trig.pi_fixed() / one == math.pi
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = trig.WORK_BITS + 20
    assert abs(mp.mpf(trig.pi_fixed()) / 2**trig.WORK_BITS - mp.pi) < mp.mpf(2) ** (-trig.WORK_BITS + 2)


def test_trig_identities_fixed_point():
    """cos^2 + sin^2 = 1 and the double-angle formulas hold to the working precision."""
    W = trig.WORK_BITS
    tol = 1 << 20  # 2^-(W-20) relative to one
    rng = np.random.default_rng(7)
    for th in list(rng.random(40) * 2 * math.pi) + [0.0, math.pi, 2 * math.pi, 1e-300]:
        for m in (1, 3, 17, 64):
            c, s = trig.cos_sin_multiple(m, th)
            assert abs(c * c + s * s - (1 << (2 * W))) < tol << W
            c2, s2 = trig.cos_sin_multiple(2 * m, th)
            assert abs(c2 - ((c * c - s * s) >> W)) < tol
            assert abs(s2 - ((2 * c * s) >> W)) < tol


def test_trig_matches_libm_within_an_ulp():
    """Small arguments where m*theta is exact in float64: libm cos/sin are within 1 ulp."""
    for th in [0.0, 0.5, 1.0, 1.5, 2.0, 3.0, 6.0, 0.1]:
        for m in (0, 1, 2, 4, 8):
            t = m * th  # exact: m is a power of two or 0 / 1
            assert abs(trig.cos_multiple(m, th) - math.cos(t)) <= math.ulp(math.cos(t))
            assert abs(trig.sin_multiple(m, th) - math.sin(t)) <= math.ulp(max(abs(math.sin(t)), 1e-300))


def test_trig_against_mpmath_correct_rounding():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 100
    rng = np.random.default_rng(11)
    for th in rng.random(50) * 2 * math.pi:
        for m in (1, 5, 33, 64, 100):
            t = mp.mpf(m) * mp.mpf(float(th))
            assert trig.cos_multiple(m, th) == float(mp.cos(t))
            assert trig.sin_multiple(m, th) == float(mp.sin(t))


def test_zernike_angular_convention():
    """Sec. 2: cos(m theta) for m >= 0, sin(|m| theta) for m < 0; Z at rho = 0 does not depend
    on theta."""
    r, th = 0.6, 0.7
    for n, m in [(4, 2), (4, -2), (5, 1), (5, -1), (6, 0)]:
        R = radial.radial(n, abs(m), r)
        ang = math.cos(abs(m) * th) if m >= 0 else math.sin(abs(m) * th)
        assert abs(basis.basis_value(n, m, r, th) - R * ang) < 1e-15
    for th in (0.1, 1.0, 4.0):
        assert basis.basis_value(4, 0, 0.0, th) == 1.0
        assert basis.basis_value(6, 2, 0.0, th) == 0.0


def test_dtheta_and_drho_against_high_precision_differences():
    """Analytic d/dtheta Z and d/drho Z against central differences of exact evaluations
    (h = 2^-30, error O(h^2))."""
    h = 2.0 ** -30
    for n, m in [(7, 3), (7, -3), (10, 0), (9, -9), (12, 4)]:
        r, th = 0.55, 2.3
        fd_t = (Fraction(basis.basis_value(n, m, r, th + h)) - Fraction(basis.basis_value(n, m, r, th - h))) / (2 * h)
        assert abs(float(fd_t) - basis.basis_dtheta(n, m, r, th)) < 1e-6
        fd_r = (radial.radial_fraction(n, m, 0, r + h) - radial.radial_fraction(n, m, 0, r - h)) / (2 * h)
        assert abs(float(fd_r) - radial.radial(n, m, r, 1)) < 1e-12


def test_basis_table_layout_and_rounding():
    ns, ms = inputs.full_zernike_modes(6)
    r, th = inputs.uniform_points(7, 3)
    zk, zt = basis.basis_table(ns, ms, r, th, 2, with_dtheta=True)
    for j in range(len(ns)):
        for p in range(len(r)):
            for k in range(3):
                assert zk[k][j][p] == basis.basis_value(int(ns[j]), int(ms[j]), r[p], th[p], k)
            assert zt[j][p] == basis.basis_dtheta(int(ns[j]), int(ms[j]), r[p], th[p])


def test_exact_sum_of_products():
    assert series.exact_sum_of_products([(1e16, 1.0), (1.0, 1.0), (-1e16, 1.0)]) == 1.0
    assert series.exact_sum_of_products([(0.1, 0.1, 10.0)]) == float(Fraction(0.1) * Fraction(0.1) * 10)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(200)
    y = rng.standard_normal(200)
    want = sum(Fraction(a) * Fraction(b) for a, b in zip(x, y))
    assert series.exact_sum_of_products(zip(x, y)) == float(want)


def test_series_against_matmul_of_basis():
    ns, ms = inputs.full_zernike_modes(8)
    r, th = inputs.uniform_points(16, 5)
    C = inputs.scaled_normal_coeffs(ns, 3, 5)
    F = np.array(series.series_eval(ns, ms, r, th, C.tolist()))
    Z = np.array(basis.basis_table(ns, ms, r, th, 0)[0][0])  # [J][P]
    assert np.max(np.abs(F - Z.T @ C)) < 1e-14


def test_adjoint_is_the_derivative_of_the_series():
    """<G, F(r, theta, C)> differentiated by central differences in exact arithmetic."""
    ns, ms = inputs.full_zernike_modes(5)
    r, th = inputs.uniform_points(4, 9)
    C = inputs.scaled_normal_coeffs(ns, 2, 9)
    G = np.random.default_rng(1).standard_normal((4, 2))
    gC, gr, gt = series.series_adjoint(ns, ms, r, th, C.tolist(), G.tolist())
    Z = np.array(basis.basis_table(ns, ms, r, th, 0)[0][0])
    assert np.max(np.abs(np.array(gC) - Z @ G)) < 1e-14

    def loss(rr, tt):
        F = series.series_eval(ns, ms, rr, tt, C.tolist())
        return sum(Fraction(F[p][s]) * Fraction(G[p, s]) for p in range(len(rr)) for s in range(2))

    h = 2.0 ** -26
    for p in range(4):
        rp, rm = r.copy(), r.copy()
        rp[p] += h
        rm[p] -= h
        assert abs(float((loss(rp, th) - loss(rm, th)) / (2 * h)) - gr[p]) < 1e-7
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        assert abs(float((loss(r, tp) - loss(r, tm)) / (2 * h)) - gt[p]) < 1e-7


def test_mixed_derivatives_against_exact_differences():
    """basis_deriv(kr, kt) against exact central differences of lower derivatives."""
    h = 2.0 ** -28
    for n, m in [(7, 3), (7, -3), (10, 0), (12, -4)]:
        r, th = 0.61, 1.7
        # d2/dtheta2 from d/dtheta
        fd = (Fraction(basis.basis_deriv(n, m, r, th + h, 0, 1)) - Fraction(basis.basis_deriv(n, m, r, th - h, 0, 1))) / (2 * h)
        assert abs(float(fd) - basis.basis_deriv(n, m, r, th, 0, 2)) < 1e-6
        # d2/drho dtheta from d/dtheta in rho
        fd = (Fraction(basis.basis_deriv(n, m, r + h, th, 0, 1)) - Fraction(basis.basis_deriv(n, m, r - h, th, 0, 1))) / (2 * h)
        assert abs(float(fd) - basis.basis_deriv(n, m, r, th, 1, 1)) < 1e-6
        # consistency with the basis table and d/dtheta
        assert basis.basis_deriv(n, m, r, th, 0, 1) == basis.basis_dtheta(n, m, r, th)
        assert basis.basis_deriv(n, m, r, th, 2, 0) == basis.basis_value(n, m, r, th, 2)


def test_point_hessian_is_the_derivative_of_the_gradient():
    """The oracle's per-point Hessian against exact central differences of its gradient."""
    ns, ms = inputs.full_zernike_modes(4)
    r, th = inputs.uniform_points(3, 12)
    C = inputs.scaled_normal_coeffs(ns, 2, 12).tolist()
    G = np.random.default_rng(4).standard_normal((3, 2)).tolist()
    gr, gt, hrr, hrt, htt = series.point_hessian(ns, ms, r, th, C, G)
    _, gr0, gt0 = series.series_adjoint(ns, ms, r, th, C, G)
    assert gr == gr0 and gt == gt0
    h = 2.0 ** -26
    for p in range(3):
        rp, rm = r.copy(), r.copy()
        rp[p] += h
        rm[p] -= h
        a = series.series_adjoint(ns, ms, rp, th, C, G)
        b = series.series_adjoint(ns, ms, rm, th, C, G)
        assert abs((a[1][p] - b[1][p]) / (2 * h) - hrr[p]) < 1e-6 * (1 + abs(hrr[p]))
        assert abs((a[2][p] - b[2][p]) / (2 * h) - hrt[p]) < 1e-6 * (1 + abs(hrt[p]))
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        a = series.series_adjoint(ns, ms, r, tp, C, G)
        b = series.series_adjoint(ns, ms, r, tm, C, G)
        assert abs((a[2][p] - b[2][p]) / (2 * h) - htt[p]) < 1e-6 * (1 + abs(htt[p]))
        assert abs((a[1][p] - b[1][p]) / (2 * h) - hrt[p]) < 1e-6 * (1 + abs(hrt[p]))  # symmetry
