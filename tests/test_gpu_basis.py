"""Parity of the CUDA Zernike-function kernel (zp_basis) with the exact oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import inputs  # noqa: E402
from oracle import basis as obasis  # noqa: E402

from helpers import assert_radial_close, radial_tolerance  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=DEV)


def check(ns, ms, r, th, kmax, with_dt=True, what=""):
    out, dt = zp.basis(ns, ms, dev(r), dev(th), kmax, dtheta=with_dt)
    got = out.cpu().numpy()
    zk, zt = obasis.basis_table(ns, ms, r, th, kmax, with_dtheta=with_dt)
    want = np.array(zk)
    for k in range(kmax + 1):
        tol = radial_tolerance(ns, k)[:, None]
        err = np.abs(got[k] - want[k])
        assert (err <= tol).all(), f"{what} k={k} max err {err.max():.3e}"
    if with_dt:
        # d/dtheta Z = |m| R (trig): bound scales with |m|
        tol = 1e-11 * np.maximum(np.abs(np.asarray(ms, dtype=np.float64)), 1.0)[:, None]
        err = np.abs(dt.cpu().numpy() - np.array(zt))
        assert (err <= tol).all(), f"{what} dtheta max err {err.max():.3e}"
    return got


def test_basis_n20_full_size():
    """Full Z set n <= 20 (231 modes), 1000 points r ~ U[0,1), theta ~ U[0,2pi): R, R', R'' times
    the angular factor and d/dtheta Z, every output element against the oracle."""
    cfg = inputs.WORKLOADS["basis_n20"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.uniform_points(cfg["n_points"], cfg["seed"])
    check(ns, ms, r, th, 2, what="basis_n20")


def test_basis_signs_origin_and_ragged():
    ns, ms = inputs.full_zernike_modes(9)
    r = np.array([0.0, 1.0, 0.5, 0.3, 0.9])
    th = np.array([0.3, 2.0, 4.0, 6.2, 1.0])
    got = check(ns, ms, r, th, 3, what="small")
    # Z at rho = 0 does not depend on theta (Sec. 2): only m = 0 modes survive
    zero_cols = got[0][:, 0]
    assert np.all(zero_cols[np.asarray(ms) != 0] == 0.0)


def test_basis_duplicates_and_large_theta():
    ns = [12, 12, 3, 12, 7]
    ms = [-4, 4, -3, -4, 1]
    r, th = inputs.uniform_points(77, 3)
    th = th * 7.0  # angles beyond 2 pi
    got = check(ns, ms, r, th, 1, what="dups")
    assert np.array_equal(got[:, 0], got[:, 3])


def test_basis_many_duplicates_per_step():
    """A mode list repeated 16 times (the Zernike x Fourier expansion of the Sec. 3 footnote):
    every step stores its value to many outputs (the angular products are formed once per
    step); each copy equals the unduplicated evaluation bit for bit, all derivatives and
    d/dtheta included, with the point tables in use (> 8192 points)."""
    ns, ms = inputs.full_zernike_modes(6)
    L = 16
    nd, md = np.repeat(ns, L), np.repeat(ms, L)
    r, th = inputs.uniform_points(9000, 44)
    rt, tt = dev(r), dev(th)
    Z1, T1 = zp.basis(ns, ms, rt, tt, 3, dtheta=True)
    Zd, Td = zp.basis(nd, md, rt, tt, 3, dtheta=True)
    torch.cuda.synchronize()
    for c in range(L):
        assert torch.equal(Zd[:, c::L, :], Z1)
        assert torch.equal(Td[c::L, :], T1)
    sub = np.array([0, 17, 4500, 8999])
    want_z, want_t = obasis.basis_table(ns, ms, r[sub], th[sub], 3, with_dtheta=True)
    got = Z1[:, :, torch.as_tensor(sub, device=DEV)].cpu().numpy()
    assert_radial_close(got, np.array(want_z), ns, "dup basis")
    assert np.max(np.abs(T1[:, torch.as_tensor(sub, device=DEV)].cpu().numpy() - np.array(want_t))) < 1e-11 * 36
