"""Per-point gradient and Hessian blocks (zp_series_point_hessian) against the oracle, and the
Hessian-vector product against differences of the GPU gradient."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import inputs  # noqa: E402
from oracle import series as oseries  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=DEV)


def test_point_hessian_against_oracle():
    ns, ms = inputs.full_zernike_modes(9)
    r, th = inputs.uniform_points(40, 31)
    r = np.concatenate([[0.0, 1.0], r])
    th = np.concatenate([[0.3, 2.0], th])
    C = inputs.scaled_normal_coeffs(ns, 3, 31)
    G = np.random.default_rng(8).standard_normal((len(r), 3))
    got = [x.cpu().numpy() for x in zp.series_point_hessian(ns, ms, dev(r), dev(th), dev(C), dev(G))]
    want = oseries.point_hessian(ns, ms, r, th, C.tolist(), G.tolist())
    scale = 1.0 + np.abs(G).sum(1) * np.abs(C).sum() * 9 ** 4
    for g, w in zip(got, want):
        assert (np.abs(g - np.array(w)) <= 1e-12 * scale).all()


def test_hvp_matches_gradient_differences():
    ns, ms = inputs.full_zernike_modes(12)
    r, th = inputs.uniform_points(500, 32)
    r = 0.05 + 0.9 * r
    C = dev(inputs.scaled_normal_coeffs(ns, 8, 32))
    G = dev(np.random.default_rng(9).standard_normal((500, 8)))
    rt, tt = dev(r), dev(th)
    plan = zp.Plan(ns, ms)
    hess = zp.series_point_hessian(None, None, rt, tt, C, G, plan=plan)
    rng = np.random.default_rng(10)
    vr, vt = dev(rng.standard_normal(500)), dev(rng.standard_normal(500))
    hv_r, hv_t = zp.series_point_hvp(None, None, rt, tt, C, G, vr, vt, plan=plan)
    # the product formed in the kernel equals the blocks applied to the tangent
    _, _, hrr, hrt, htt = hess
    assert float((hv_r - (hrr * vr + hrt * vt)).abs().max()) <= 1e-13 * (1 + float(hv_r.abs().max()))
    assert float((hv_t - (hrt * vr + htt * vt)).abs().max()) <= 1e-13 * (1 + float(hv_t.abs().max()))
    eps = 1e-6
    gp = zp.series_point_hessian(None, None, rt + eps * vr, tt + eps * vt, C, G, plan=plan)
    gm = zp.series_point_hessian(None, None, rt - eps * vr, tt - eps * vt, C, G, plan=plan)
    fd_r = (gp[0] - gm[0]) / (2 * eps)
    fd_t = (gp[1] - gm[1]) / (2 * eps)
    assert float((fd_r - hv_r).abs().max()) < 1e-5 * (1 + float(hv_r.abs().max()))
    assert float((fd_t - hv_t).abs().max()) < 1e-5 * (1 + float(hv_t.abs().max()))
    # the gradient part equals the adjoint's to float64 accuracy (the adjoint's default takes
    # the point gradients of at most 16 sets from the fused kernel's derivative series, the
    # Hessian kernel from H = C G^T)
    _, gr, gt = zp.series_adjoint(None, None, rt, tt, C, G, plan=plan)
    for a, b in ((gr, hess[0]), (gt, hess[1])):
        assert float((a - b).abs().max()) <= 1e-12 * (1 + float(b.abs().max()))
