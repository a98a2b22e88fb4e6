"""Least-squares fit (zp_series_fit) against the oracle fit and the known-coefficient limit."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import inputs  # noqa: E402
from oracle import fit as ofit  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=DEV)


def polar_quadrature(n_r, n_theta):
    r, th = inputs.polar_grid(n_r, n_theta)
    _, wgl = np.polynomial.legendre.leggauss(n_r)
    return r, th, np.repeat(0.25 * wgl, n_theta) * (2.0 * math.pi / n_theta)


def test_weighted_fit_against_oracle():
    ns, ms = inputs.full_zernike_modes(10)
    r, th, w = polar_quadrature(12, 24)
    Y = np.random.default_rng(1).standard_normal((len(r), 5))
    got = zp.series_fit(ns, ms, dev(r), dev(th), dev(Y), weights=dev(w)).cpu().numpy()
    want = ofit.series_fit(ns, ms, r, th, Y, w)
    assert np.max(np.abs(got - want)) < 1e-10 * (1 + np.max(np.abs(want)))


def test_unweighted_and_ridge_fit_against_oracle():
    ns = [5, 3, 3, 0, 8, 7]
    ms = [1, -3, 3, 0, -4, 7]
    r, th = inputs.uniform_points(200, 3)
    Y = np.random.default_rng(2).standard_normal((200, 3))
    for ridge in (0.0, 0.5):
        got = zp.series_fit(ns, ms, dev(r), dev(th), dev(Y), ridge=ridge).cpu().numpy()
        want = ofit.series_fit(ns, ms, r, th, Y, ridge=ridge)
        assert np.max(np.abs(got - want)) < 1e-10 * (1 + np.max(np.abs(want)))


def test_fit_recovers_series_n24_coefficients_at_full_size():
    """Samples of a known series on the 325-mode, 250 x 200 polar grid with 256 sets: the fit
    returns the coefficients (round trip through zp_series_eval)."""
    cfg = inputs.WORKLOADS["series_n24"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th, w = polar_quadrature(cfg["n_r"], cfg["n_theta"])
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    plan = zp.Plan(ns, ms)
    rt, tt = dev(r), dev(th)
    Y = zp.series_eval(None, None, rt, tt, dev(C), plan=plan)
    got = zp.series_fit(None, None, rt, tt, Y, weights=dev(w), plan=plan).cpu().numpy()
    assert np.max(np.abs(got - C)) < 1e-10


def test_singular_fit_is_reported_and_ridge_fixes_it():
    ns, ms = inputs.full_zernike_modes(4)  # 15 modes
    r, th = inputs.uniform_points(3, 9)  # 3 points: rank-deficient normal matrix
    Y = np.ones((3, 2))
    with pytest.raises(zp.ZernikeError) as e:
        zp.series_fit(ns, ms, dev(r), dev(th), dev(Y))
    assert "positive definite" in str(e.value)
    C = zp.series_fit(ns, ms, dev(r), dev(th), dev(Y), ridge=1e-3)
    assert bool(torch.isfinite(C).all())


@pytest.mark.parametrize("n_max,S", [(7, 3), (34, 5), (35, 1), (44, 33)])
def test_fit_round_trip_across_solver_sizes(n_max, S):
    """Round trips through zp_series_eval on an exact polar quadrature for 36 modes (two
    32-column panels, ragged), 630 modes (the one-kernel solve near its 640-mode shared-memory
    limit), 666 and 1035 modes (beyond it: the blocked triangular solves, ragged blocks and more
    than 32 right-hand sides), with odd set counts."""
    ns, ms = inputs.full_zernike_modes(n_max)
    r, th, w = polar_quadrature(n_max // 2 + 3, 2 * n_max + 4)
    C = np.random.default_rng(n_max).standard_normal((len(ns), S))
    plan = zp.Plan(ns, ms)
    rt, tt = dev(r), dev(th)
    Y = zp.series_eval(None, None, rt, tt, dev(C), plan=plan)
    for prec in ("fp64", "fp64emu"):
        got = zp.series_fit(None, None, rt, tt, Y, weights=dev(w), plan=plan, prec=prec).cpu().numpy()
        assert np.max(np.abs(got - C)) < 1e-9, (prec, np.max(np.abs(got - C)))
