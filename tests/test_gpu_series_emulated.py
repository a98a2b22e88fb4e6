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


@pytest.mark.parametrize("nmax", [24, 32, 60, 100])
def test_emulated_fp64_one_batch_plane_shapes(nmax):
    """Outputs large enough for one K batch (>= 304 point tiles) with each slice width: the
    paired planes (4, 5, 6 and 7 of them for beta = 7, 6, 5, 4) and the fully unrolled
    recombination of each shape, against the DGEMM float64 path everywhere."""
    ns, ms = inputs.full_zernike_modes(nmax)
    r, th = inputs.sqrt_uniform_points(40_000, 71 + nmax)
    C = inputs.scaled_normal_coeffs(ns, 20, 71 + nmax)
    plan = zp.Plan(ns, ms)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    F = zp.series_eval(None, None, rt, tt, Ct, "fp64emu", plan=plan)
    F64 = zp.series_eval(None, None, rt, tt, Ct, "fp64", plan=plan)
    Z = zp.basis(None, None, rt, tt, 0, plan=plan)[0][0].abs()
    bound = 2e-13 * (1.0 + Z.T @ Ct.abs())
    assert bool(((F - F64).abs() <= bound).all())


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


def scale_bound(K, A_rows, B_rows):
    """The slicing scheme's bound for C[m][n] = sum_k A[m][k] B[n][k]: every operand is cut to
    54 bits of its row's power-of-two scale, so the error is about K 2^-54 max_k |A[m]|
    max_k |B[n]|; 2^-48 leaves a factor 64 of slack."""
    return K * 2.0 ** -48 * np.outer(np.abs(A_rows).max(axis=1), np.abs(B_rows).max(axis=1))


@pytest.mark.parametrize("nmax,P,S", [(7, 90, 4), (3, 1500, 3)])
def test_emulated_adjoint_against_oracle(nmax, P, S):
    """grad_C = Z G (contraction over the points; 1500 points with 10 modes cut K into many
    batches) by the emulated contraction, grad_r and grad_theta (at most 16 sets) as row sums
    of G times the fused kernel's derivative series."""
    ns, ms = inputs.full_zernike_modes(nmax)
    r, th = inputs.uniform_points(P, 22 + nmax)
    C = inputs.scaled_normal_coeffs(ns, S, 22)
    G = np.random.default_rng(5).standard_normal((P, S))
    gC, gr, gt = zp.series_adjoint(ns, ms, dev(r), dev(th), dev(C), dev(G), prec="fp64emu")
    wC, wr, wt = oseries.series_adjoint(ns, ms, r, th, C.tolist(), G.tolist())
    Z = np.array(obasis.basis_table(ns, ms, r, th, 0)[0][0])  # [J][P]
    tolC = 1e-13 * (1.0 + np.abs(Z) @ np.abs(G)) + scale_bound(P, Z, G.T)
    assert (np.abs(gC.cpu().numpy() - np.array(wC)) <= tolC).all()
    scale = 1.0 + np.abs(G).sum(1) * np.abs(C).sum() * max(nmax, 1) ** 2
    assert (np.abs(gr.cpu().numpy() - np.array(wr)) <= 1e-12 * scale).all()
    assert (np.abs(gt.cpu().numpy() - np.array(wt)) <= 1e-12 * scale).all()


@pytest.mark.parametrize("S", [1, 16, 17])
def test_emulated_adjoint_point_gradients_off_disc(S):
    """Points inside and beyond the unit disc (r up to 1.4), one to 17 sets (17: through H =
    C G^T instead of the fused derivative series): grad_r and grad_theta against the float64
    DGEMM form, relative to the size of the terms they sum."""
    ns, ms = inputs.full_zernike_modes(15)
    rng = np.random.default_rng(80 + S)
    P = 700
    r, th = rng.uniform(0.0, 1.4, P), rng.uniform(-np.pi, np.pi, P)
    C = inputs.scaled_normal_coeffs(ns, S, 80 + S)
    G = rng.standard_normal((P, S))
    args = (ns, ms, dev(r), dev(th), dev(C), dev(G))
    gc, gr, gt = zp.series_adjoint(*args, prec="fp64emu")
    wc, wr, wt = zp.series_adjoint(*args, prec="fp64")
    scale = 1.0 + torch.as_tensor(np.abs(G).sum(1) * np.abs(C).sum() * 15 ** 2 * r.max() ** 15, device=DEV)
    assert bool(((gr - wr).abs() <= 1e-12 * scale).all())
    assert bool(((gt - wt).abs() <= 1e-12 * scale).all())
    # grad_C = Z G with Z's row scales from the walk's row maxima (|Z| up to about 1.4^15 here):
    # within K 2^-54 max_p |Z_j(p)| sum_p |G[p][s]| of the DGEMM form.
    Z = zp.basis(ns, ms, dev(r), dev(th))[0][0]
    zmax = Z.abs().max(dim=1).values[:, None]
    gsum = torch.as_tensor(np.abs(G).sum(0), device=DEV)[None, :]
    assert bool(((gc - wc).abs() <= 1e-13 * (1.0 + zmax * gsum)).all())


def test_emulated_adjoint_series_n24_full_size_against_fp64():
    """The 325-mode, 50000-point, 256-set adjoint: the emulated contractions (grad_C over 50000
    points in K batches, H over 256 sets) against the DGEMM path."""
    cfg = inputs.WORKLOADS["series_n24"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.polar_grid(cfg["n_r"], cfg["n_theta"])
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    plan = zp.Plan(ns, ms)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    G = torch.randn((len(r), C.shape[1]), dtype=torch.float64, device=DEV,
                    generator=torch.Generator(DEV).manual_seed(3))
    e = zp.series_adjoint(None, None, rt, tt, Ct, G, plan=plan, prec="fp64emu")
    f = zp.series_adjoint(None, None, rt, tt, Ct, G, plan=plan, prec="fp64")
    Z = zp.basis(None, None, rt, tt, 0, plan=plan)[0][0]
    bC = 1e-12 * (1.0 + Z.abs() @ G.abs()) + len(r) * 2.0 ** -48 * torch.outer(Z.abs().amax(1), G.abs().amax(0))
    assert bool(((e[0] - f[0]).abs() <= bC).all())
    for a, b in zip(e[1:], f[1:]):
        assert bool(((a - b).abs() <= 1e-10 * (1.0 + b.abs().max())).all())


def test_emulated_fit_against_oracle_and_fp64():
    """Weighted least squares with the Gram matrix and right-hand side by the emulated
    contraction: against the oracle fit, and the full-size series_n24 round trip."""
    from oracle import fit as ofit

    ns, ms = inputs.full_zernike_modes(10)
    r, th = inputs.polar_grid(12, 24)
    _, wgl = np.polynomial.legendre.leggauss(12)
    w = np.repeat(0.25 * wgl, 24) * (2.0 * np.pi / 24)
    Y = np.random.default_rng(1).standard_normal((len(r), 5))
    got = zp.series_fit(ns, ms, dev(r), dev(th), dev(Y), weights=dev(w), prec="fp64emu").cpu().numpy()
    want = ofit.series_fit(ns, ms, r, th, Y, w)
    assert np.max(np.abs(got - want)) < 1e-10 * (1 + np.max(np.abs(want)))
    cfg = inputs.WORKLOADS["series_n24"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.polar_grid(cfg["n_r"], cfg["n_theta"])
    _, wgl = np.polynomial.legendre.leggauss(cfg["n_r"])
    w = np.repeat(0.25 * wgl, cfg["n_theta"]) * (2.0 * np.pi / cfg["n_theta"])
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    plan = zp.Plan(ns, ms)
    rt, tt = dev(r), dev(th)
    Yf = zp.series_eval(None, None, rt, tt, dev(C), plan=plan)
    got = zp.series_fit(None, None, rt, tt, Yf, weights=dev(w), plan=plan, prec="fp64emu").cpu().numpy()
    assert np.max(np.abs(got - C)) < 1e-10


def test_emulated_autograd_matches_fp64_autograd():
    """zernike_series with prec="fp64emu" runs the emulated forward and adjoint; its gradients
    for r, theta and C agree with the DGEMM path's."""
    ns, ms = inputs.full_zernike_modes(9)
    r, th = inputs.uniform_points(400, 31)
    C = inputs.scaled_normal_coeffs(ns, 6, 31)
    plan = zp.Plan(ns, ms)
    W = torch.randn((400, 6), dtype=torch.float64, device=DEV, generator=torch.Generator(DEV).manual_seed(9))
    grads = []
    for prec in ("fp64", "fp64emu"):
        rt, tt, Ct = (dev(x).requires_grad_() for x in (r, th, C))
        F = zp.zernike_series(rt, tt, Ct, plan, prec=prec)
        (F * W).sum().backward()
        grads.append((F.detach(), rt.grad, tt.grad, Ct.grad))
    for a, b in zip(grads[0], grads[1]):
        assert bool(((a - b).abs() <= 1e-11 * (1.0 + b.abs().max())).all())


def test_emulated_non_finite_inputs_give_nan_rows_and_sets():
    """An infinity or NaN in a coefficient set makes that set's outputs NaN, a NaN point makes
    that point's outputs NaN; every other output keeps float64 accuracy."""
    ns, ms = inputs.full_zernike_modes(6)
    r, th = inputs.uniform_points(300, 12)
    r[7] = np.nan
    C = inputs.scaled_normal_coeffs(ns, 5, 12)
    C[3, 1] = np.nan
    C[0, 2] = np.inf
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), "fp64emu").cpu().numpy()
    assert np.isnan(F[:, 1]).all() and np.isnan(F[:, 2]).all() and np.isnan(F[7]).all()
    ok_rows = np.array([p for p in range(300) if p != 7])
    good = np.ix_(ok_rows, [0, 3, 4])
    Cg = C[:, [0, 3, 4]]
    want = np.array(oseries.series_eval(ns, ms, r[ok_rows], th[ok_rows], Cg.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r[ok_rows], th[ok_rows], Cg))
    assert (np.abs(F[good] - want) <= tol).all()


@pytest.mark.parametrize("S", [1, 7, 16])
def test_stacked_diagonals_match_plane_launches(S, monkeypatch):
    """A narrow B (at most 16 sets) takes the stacked-diagonal slice products (one launch forms
    every diagonal); ZP_EMU_STACKED=0 takes the launch per plane of paired diagonals.  Both form
    the same exact integer sums, so grad_C over a long K (30000 points, many K batches) and a
    forward whose K (5151 modes) is past the fused kernel's limit agree bitwise, and with the
    DGEMM form to the float64 tolerance."""
    ns, ms = inputs.full_zernike_modes(20)
    rng = np.random.default_rng(90 + S)
    P = 30000
    r, th = np.sqrt(rng.uniform(0.0, 1.0, P)), rng.uniform(0.0, 2 * np.pi, P)
    C = inputs.scaled_normal_coeffs(ns, S, 90 + S)
    G = rng.standard_normal((P, S))
    args = (ns, ms, dev(r), dev(th), dev(C), dev(G))
    gc = zp.series_adjoint(*args, prec="fp64emu")[0]
    monkeypatch.setenv("ZP_EMU_STACKED", "0")
    gc_planes = zp.series_adjoint(*args, prec="fp64emu")[0]
    monkeypatch.delenv("ZP_EMU_STACKED")
    assert torch.equal(gc, gc_planes)
    want = zp.series_adjoint(*args, prec="fp64")[0]
    scale = 1.0 + torch.as_tensor(np.abs(G).sum(0), device=DEV)[None, :]
    assert bool(((gc - want).abs() <= 1e-13 * scale).all())

    ns2, ms2 = inputs.full_zernike_modes(100)
    P2 = 600
    r2, th2 = rng.uniform(0.0, 1.0, P2), rng.uniform(0.0, 2 * np.pi, P2)
    C2 = inputs.scaled_normal_coeffs(ns2, S, 91 + S)
    a2 = (ns2, ms2, dev(r2), dev(th2), dev(C2))
    F = zp.series_eval(*a2, "fp64emu")
    monkeypatch.setenv("ZP_EMU_STACKED", "0")
    F_planes = zp.series_eval(*a2, "fp64emu")
    monkeypatch.delenv("ZP_EMU_STACKED")
    assert torch.equal(F, F_planes)
    F64 = zp.series_eval(*a2, "fp64")
    scale2 = 1.0 + torch.as_tensor(np.abs(C2).sum(0), device=DEV)[None, :]
    assert bool(((F - F64).abs() <= 1e-13 * scale2).all())


def test_stacked_diagonals_widest_slices(monkeypatch):
    """1.6 million points and two sets: grad_C's K is long enough that the slice width drops to
    5 bits (11 slices, the widest stacked MMA, N = 176); stacked and plane launches agree
    bitwise, and both with the DGEMM form to the float64 tolerance."""
    ns, ms = inputs.full_zernike_modes(4)
    rng = np.random.default_rng(97)
    P, S = 1_600_000, 2
    r, th = np.sqrt(rng.uniform(0.0, 1.0, P)), rng.uniform(0.0, 2 * np.pi, P)
    C = inputs.scaled_normal_coeffs(ns, S, 97)
    G = rng.standard_normal((P, S))
    args = (ns, ms, dev(r), dev(th), dev(C), dev(G))
    gc = zp.series_adjoint(*args, need=(True, False, False), prec="fp64emu")[0]
    monkeypatch.setenv("ZP_EMU_STACKED", "0")
    gc_planes = zp.series_adjoint(*args, need=(True, False, False), prec="fp64emu")[0]
    monkeypatch.delenv("ZP_EMU_STACKED")
    assert torch.equal(gc, gc_planes)
    want = zp.series_adjoint(*args, need=(True, False, False), prec="fp64")[0]
    scale = 1.0 + torch.as_tensor(np.abs(G).sum(0), device=DEV)[None, :]
    assert bool(((gc - want).abs() <= 1e-13 * scale).all())
