"""Pins of the oracle's least-squares fit: quadrature orthogonality (closed-form norms),
recovery of known coefficients, and the ridge limit."""
import math

import numpy as np

from oracle import fit as ofit, series as oseries
from paper_2409_19156_gb300 import inputs


def polar_quadrature(n_r, n_theta):
    """Polar grid (Gauss-Legendre in r^2, uniform theta) and weights that integrate
    f(rho, theta) rho drho dtheta over the disc exactly for polynomial Zernike products."""
    r, th = inputs.polar_grid(n_r, n_theta)
    _, wgl = np.polynomial.legendre.leggauss(n_r)
    w = np.repeat(0.25 * wgl, n_theta) * (2.0 * math.pi / n_theta)
    return r, th, w


def test_quadrature_gram_is_diagonal_with_closed_form_norms():
    """int Z_j Z_j' rho drho dtheta = delta_jj' * pi / (2(n+1)) (m != 0), pi / (n+1) (m = 0)."""
    ns, ms = inputs.full_zernike_modes(8)
    r, th, w = polar_quadrature(12, 24)
    A, _ = ofit.normal_matrix(ns, ms, r, th, w)
    want = np.diag([math.pi / (2 * (n + 1)) if m != 0 else math.pi / (n + 1) for n, m in zip(ns, ms)])
    assert np.max(np.abs(A - want)) < 1e-14


def test_fit_recovers_known_coefficients():
    ns, ms = inputs.full_zernike_modes(6)
    r, th = inputs.uniform_points(120, 4)
    C = inputs.scaled_normal_coeffs(ns, 3, 4)
    Y = np.array(oseries.series_eval(ns, ms, r, th, C.tolist()))
    got = ofit.series_fit(ns, ms, r, th, Y)
    assert np.max(np.abs(got - C)) < 1e-11


def test_ridge_limit():
    ns, ms = inputs.full_zernike_modes(3)
    r, th = inputs.uniform_points(30, 5)
    Y = np.random.default_rng(0).standard_normal((30, 2))
    lam = 1e12
    _, Z = ofit.normal_matrix(ns, ms, r, th)
    got = ofit.series_fit(ns, ms, r, th, Y, ridge=lam)
    assert np.max(np.abs(got * lam - Z @ Y)) < 1e-6 * np.max(np.abs(Z @ Y))
