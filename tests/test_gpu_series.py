"""Parity of the float64 series and its adjoint (zp_series_eval / zp_series_adjoint) with the
oracle, and the autograd wrapper against central finite differences.  The default float64 path
is the emulated tensor-core contraction; the small cases also run the DGEMM baseline."""
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


def abs_bound(ns, ms, r, th, C, G=None):
    """Sum of |terms| of each output: the scale of the float64 rounding bound."""
    Z = np.abs(np.array(obasis.basis_table(ns, ms, r, th, 0)[0][0]))  # [J][P]
    if G is None:
        return Z.T @ np.abs(C)  # [P][S]
    return Z @ np.abs(G)  # [J][S]


@pytest.mark.parametrize("prec", ["fp64emu", "fp64"])
def test_series_eval_fp64_small(prec):
    ns, ms = inputs.full_zernike_modes(8)
    r, th = inputs.uniform_points(300, 21)
    C = inputs.scaled_normal_coeffs(ns, 5, 21)
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), prec).cpu().numpy()
    want = np.array(oseries.series_eval(ns, ms, r, th, C.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r, th, C))
    assert (np.abs(F - want) <= tol).all()


@pytest.mark.parametrize("prec", ["fp64emu", "fp64"])
def test_series_adjoint_fp64_small(prec):
    ns, ms = inputs.full_zernike_modes(7)
    r, th = inputs.uniform_points(90, 22)
    C = inputs.scaled_normal_coeffs(ns, 4, 22)
    G = np.random.default_rng(5).standard_normal((90, 4))
    gC, gr, gt = zp.series_adjoint(ns, ms, dev(r), dev(th), dev(C), dev(G), prec=prec)
    wC, wr, wt = oseries.series_adjoint(ns, ms, r, th, C.tolist(), G.tolist())
    tolC = 1e-13 * (1.0 + abs_bound(ns, ms, r, th, C, G))
    assert (np.abs(gC.cpu().numpy() - np.array(wC)) <= tolC).all()
    scale = 1.0 + np.abs(G).sum(1) * np.abs(C).sum() * 7 ** 2  # |dZ/drho| <= n^2-ish, |dZ/dtheta| <= n
    assert (np.abs(gr.cpu().numpy() - np.array(wr)) <= 1e-12 * scale).all()
    assert (np.abs(gt.cpu().numpy() - np.array(wt)) <= 1e-12 * scale).all()
    # Outputs may be requested individually
    gC2, gr2, gt2 = zp.series_adjoint(ns, ms, dev(r), dev(th), dev(C), dev(G), need=(False, True, False), prec=prec)
    assert gC2 is None and gt2 is None
    assert torch.equal(gr2, gr)


def test_series_n24_polar_grid_sampled():
    """The 325-mode, 250x200 polar-grid, 256-set workload at full size; sampled rows against
    the oracle (exact sums over the oracle basis)."""
    cfg = inputs.WORKLOADS["series_n24"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.polar_grid(cfg["n_r"], cfg["n_theta"])
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    plan = zp.Plan(ns, ms)
    F = zp.series_eval(None, None, dev(r), dev(th), dev(C), plan=plan)
    rows = np.array([0, 1, 199, 200, 24_999, 49_999, 31_337])
    got = F[torch.as_tensor(rows, device=DEV)].cpu().numpy()
    want = np.array(oseries.series_eval(ns, ms, r[rows], th[rows], C.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r[rows], th[rows], C))
    assert (np.abs(got - want) <= tol).all()


def test_autograd_matches_central_differences():
    """spec check: d<G, F>/d(C, r, theta) from the adjoint vs central differences, h = 1e-6."""
    ns, ms = inputs.full_zernike_modes(10)
    r, th = inputs.uniform_points(40, 23)
    r = 0.05 + 0.9 * r  # keep r +- h inside the disc's interior
    C = inputs.scaled_normal_coeffs(ns, 3, 23)
    G = dev(np.random.default_rng(6).standard_normal((40, 3)))
    plan = zp.Plan(ns, ms)
    rt = dev(r).requires_grad_(True)
    tt = dev(th).requires_grad_(True)
    Ct = dev(C).requires_grad_(True)
    F = zp.zernike_series(rt, tt, Ct, plan)
    (F * G).sum().backward()
    h = 1e-6

    def loss(rr, t2, cc):
        return float((zp.series_eval(None, None, rr, t2, cc, plan=plan) * G).sum())

    base_r, base_t, base_C = dev(r), dev(th), dev(C)
    for p in (0, 7, 39):
        e = torch.zeros(40, dtype=torch.float64, device=DEV)
        e[p] = h
        fd = (loss(base_r + e, base_t, base_C) - loss(base_r - e, base_t, base_C)) / (2 * h)
        assert abs(fd - float(rt.grad[p])) < 1e-6 * (1 + abs(fd))
        fd = (loss(base_r, base_t + e, base_C) - loss(base_r, base_t - e, base_C)) / (2 * h)
        assert abs(fd - float(tt.grad[p])) < 1e-6 * (1 + abs(fd))
    for j, s in ((0, 0), (17, 2), (len(ns) - 1, 1)):
        e = torch.zeros_like(base_C)
        e[j, s] = h
        fd = (loss(base_r, base_t, base_C + e) - loss(base_r, base_t, base_C - e)) / (2 * h)
        assert abs(fd - float(Ct.grad[j, s])) < 1e-6 * (1 + abs(fd))


def test_series_empty_and_errors():
    ns, ms = inputs.full_zernike_modes(3)
    r, th = inputs.uniform_points(5, 1)
    C = np.ones((len(ns), 0))
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C))
    assert F.shape == (5, 0)
    with pytest.raises(ValueError):
        zp.series_eval(ns, ms, dev(r), dev(th), dev(np.ones((3, 2))))


def test_series_n24_full_size_autograd_against_central_differences():
    """The 325-mode, 50000-point polar-grid, 256-set workload through the autograd wrapper:
    sampled gradient entries (r, theta, C) against central differences with h = 1e-6."""
    cfg = inputs.WORKLOADS["series_n24"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.polar_grid(cfg["n_r"], cfg["n_theta"])
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    plan = zp.Plan(ns, ms)
    G = torch.randn((len(r), C.shape[1]), dtype=torch.float64, device=DEV,
                    generator=torch.Generator(DEV).manual_seed(3))
    rt = dev(r).requires_grad_(True)
    tt = dev(th).requires_grad_(True)
    Ct = dev(C).requires_grad_(True)
    (zp.zernike_series(rt, tt, Ct, plan) * G).sum().backward()
    h = 1e-6
    base = (dev(r), dev(th), dev(C))

    # Perturbing r_p or theta_p changes only row p of F, and C[j, s] only column s, so the
    # finite-difference loss sums just that row / column (summing all 1.28e7 products would
    # put ~1e-9 of rounding noise into each loss value, 5e-4 after dividing by 2h).
    def row_loss(p, rr, t2, cc):
        F = zp.series_eval(None, None, rr, t2, cc, plan=plan)
        return float((F[p] * G[p]).sum())

    def col_loss(s, rr, t2, cc):
        F = zp.series_eval(None, None, rr, t2, cc, plan=plan)
        return float((F[:, s] * G[:, s]).sum())

    for p in (0, 12_345, 49_999):
        for which, grad in ((0, rt.grad), (1, tt.grad)):
            e = torch.zeros(len(r), dtype=torch.float64, device=DEV)
            e[p] = h
            plus = list(base)
            minus = list(base)
            plus[which] = base[which] + e
            minus[which] = base[which] - e
            fd = (row_loss(p, *plus) - row_loss(p, *minus)) / (2 * h)
            assert abs(fd - float(grad[p])) < 1e-6 * (1 + abs(fd)), (which, p, fd, float(grad[p]))
    for j, s in ((0, 0), (200, 100), (324, 255)):
        e = torch.zeros_like(base[2])
        e[j, s] = h
        fd = (col_loss(s, base[0], base[1], base[2] + e) - col_loss(s, base[0], base[1], base[2] - e)) / (2 * h)
        assert abs(fd - float(Ct.grad[j, s])) < 1e-6 * (1 + abs(fd))
