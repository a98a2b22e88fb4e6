"""Float64-accurate series on the tensor cores (zp_series_eval with ZP_PREC_FP64_EMULATED):
the same float64 tolerance as the DGEMM path, against the exact oracle and the DGEMM path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import inputs  # noqa: E402
from oracle import basis as obasis, series as oseries  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=DEV)


def abs_bound(ns, ms, r, th, C):
    Z = np.abs(np.array(obasis.basis_table(ns, ms, r, th, 0)[0][0]))
    return Z.T @ np.abs(C)


@pytest.mark.parametrize("nmax,P,S", [(8, 300, 5), (3, 1, 1), (12, 129, 300), (0, 4, 2)])
def test_emulated_fp64_against_oracle(nmax, P, S):
    ns, ms = inputs.full_zernike_modes(nmax)
    r, th = inputs.uniform_points(P, 50 + nmax)
    if P > 2:
        r[:2] = [0.0, 1.0]  # a row that is zero except for m = 0 modes, and the unit circle
    C = inputs.scaled_normal_coeffs(ns, S, 50 + nmax) * 37.5
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), "fp64emu").cpu().numpy()
    assert F.dtype == np.float64
    want = np.array(oseries.series_eval(ns, ms, r, th, C.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r, th, C))
    assert (np.abs(F - want) <= tol).all(), float(np.max(np.abs(F - want) / tol))


@pytest.mark.parametrize("nmax", [40, 60, 100])
def test_emulated_fp64_narrower_slices(nmax):
    """861 / 1891 / 5151 modes (padded K 896 / 1920 / 5184) take the beta = 6, 5 and 4 slice
    widths (9, 11 and 14 slices) that keep every float32 partial sum exact."""
    ns, ms = inputs.full_zernike_modes(nmax)
    r, th = inputs.sqrt_uniform_points(200, 61)
    C = inputs.scaled_normal_coeffs(ns, 20, 61)
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), "fp64emu").cpu().numpy()
    rows = [0, 77, 199]
    want = np.array(oseries.series_eval(ns, ms, r[rows], th[rows], C.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r[rows], th[rows], C))
    assert (np.abs(F[rows] - want) <= tol).all()


def test_emulated_fp64_series_n24_full_size():
    """The 325-mode, 50000-point polar grid, 256 sets: against the DGEMM float64 path everywhere
    and against the oracle on sampled rows."""
    cfg = inputs.WORKLOADS["series_n24"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.polar_grid(cfg["n_r"], cfg["n_theta"])
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    plan = zp.Plan(ns, ms)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    F = zp.series_eval(None, None, rt, tt, Ct, "fp64emu", plan=plan)
    F64 = zp.series_eval(None, None, rt, tt, Ct, "fp64", plan=plan)
    Z = zp.basis(None, None, rt, tt, 0, plan=plan)[0][0].abs()
    bound = 2e-13 * (1.0 + Z.T @ Ct.abs())
    assert bool(((F - F64).abs() <= bound).all())
    rows = np.array([0, 199, 24_999, 49_999])
    want = np.array(oseries.series_eval(ns, ms, r[rows], th[rows], C.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r[rows], th[rows], C))
    assert (np.abs(F[torch.as_tensor(rows, device=DEV)].cpu().numpy() - want) <= tol).all()


def test_emulated_fp64_extreme_column_scales():
    """Coefficient sets scaled by 2^300, 2^-300 and 2^-1000, an all-zero set and one dominant
    coefficient: the power-of-two scales and the final rounding keep float64 accuracy.  Set 4
    (one coefficient 1e10 beside entries of order 1) is held to the scheme's scale-relative
    bound: every operand is cut to 54 bits of its row / column scale, so F[p][s] is exact to
    about J 2^-54 max_j |Z[j][p]| max_j |C[j][s]| (2^-48 leaves a factor 64 of slack)."""
    ns, ms = inputs.full_zernike_modes(10)
    r, th = inputs.uniform_points(150, 71)
    C = inputs.scaled_normal_coeffs(ns, 6, 71)
    C[:, 0] *= 2.0 ** 300
    C[:, 1] *= 2.0 ** -300
    C[:, 2] = 0.0
    C[:, 3] *= 2.0 ** -1000
    C[5, 4] = 1e10
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), "fp64emu").cpu().numpy()
    want = np.array(oseries.series_eval(ns, ms, r, th, C.tolist()))
    Z = np.abs(np.array(obasis.basis_table(ns, ms, r, th, 0)[0][0]))
    scale_bound = len(ns) * 2.0 ** -48 * np.outer(Z.max(axis=0), np.abs(C).max(axis=0))
    tol = 1e-13 * abs_bound(ns, ms, r, th, C) + 1e-320
    tol[:, 4] += scale_bound[:, 4]
    assert (F[:, 2] == 0.0).all()
    assert (np.abs(F - want) <= tol).all(), float(np.max(np.abs(F - want) / tol))
