"""Parity of the CUDA recursion walk (zp_radial / zp_radial_per_mode) with the exact oracle."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import _lib, inputs  # noqa: E402
from oracle import radial as oradial  # noqa: E402

from helpers import assert_radial_close  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=DEV)


def run_radial(ns, ms, r, kmax, plan=False):
    rt = dev(r)
    if plan:
        p = zp.Plan(ns, ms)
        out = zp.radial(None, None, rt, kmax, plan=p)
    else:
        out = zp.radial(ns, ms, rt, kmax)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_small_full_radial_set_all_derivatives():
    """Every radial mode n <= 12 at points including 0, 1 and exactly representable ones."""
    ns, ms = inputs.radial_modes(12)
    r = np.concatenate([[0.0, 1.0, 0.5, 0.25, 0.75, 0.125], inputs.uniform_points(58, 100)[0]])
    got = run_radial(ns, ms, r, 3)
    want = np.array(oradial.radial_table(ns, ms, r, 3))
    assert_radial_close(got, want, ns, "n<=12")
    # k = 0 values at r = 1 are exactly 1 up to rounding of the recursion
    assert np.max(np.abs(got[0][:, 1] - 1.0)) < 1e-13


def test_fig1_protocol_n50_linspace():
    """Sec. 4 accuracy protocol: 100 linearly spaced rho, all (n, m) with n, m <= 50, k = 0..3.
    The paper reports a largest error of 2.05e-14 for its float64 recursion (k = 0)."""
    ns, ms = inputs.radial_modes(50)
    r = inputs.linspace_points(100)
    got = run_radial(ns, ms, r, 3, plan=True)
    want = np.array(oradial.radial_table(ns, ms, r, 3))
    stats = assert_radial_close(got, want, ns, "fig1")
    assert stats[0] < 1e-13, stats


def test_radial_n100_full_size_sampled_points():
    """The 2601-mode, 100000-point Chebyshev-Gauss workload in the benchmark's launch
    configuration; outputs compared on sampled points (all modes, k = 0..3)."""
    ns, ms = inputs.radial_modes(100)
    r = inputs.chebyshev_gauss_points(100_000)
    rt = dev(r)
    plan = zp.Plan(ns, ms)
    out = zp.radial(None, None, rt, 3, plan=plan)
    rng = np.random.default_rng(123)
    pts = np.unique(np.concatenate([[0, 1, 99_998, 99_999], rng.integers(0, 100_000, 40)]))
    got = out[:, :, torch.as_tensor(pts, device=DEV)].cpu().numpy()
    want = np.array(oradial.radial_table(ns, ms, r[pts], 3))
    assert_radial_close(got, want, ns, "n<=100")
    assert np.isfinite(out.cpu().numpy()).all()


@pytest.mark.parametrize("P", [1, 2, 3, 255, 256, 257, 1001])
def test_ragged_point_counts(P):
    ns, ms = inputs.radial_modes(16)
    r = inputs.uniform_points(P, 7)[0]
    got = run_radial(ns, ms, r, 2)
    want = np.array(oradial.radial_table(ns, ms, r, 2))
    assert_radial_close(got, want, ns, f"P={P}")


def test_duplicated_scrambled_and_sparse_modes():
    """Caller order, duplicated modes (Sec. 3 footnote) and sparse columns (gaps in N)."""
    ns = [30, 4, 4, 9, 30, 0, 17, 4, 22]
    ms = [0, 2, -2, 9, -4, 0, 1, 2, 22]
    r = inputs.uniform_points(100, 8)[0]
    got = run_radial(ns, ms, r, 3)
    want = np.array(oradial.radial_table(ns, ms, r, 3))
    assert_radial_close(got, want, ns, "scrambled")
    assert np.array_equal(got[:, 1], got[:, 2]) and np.array_equal(got[:, 1], got[:, 7])


def test_points_outside_unit_interval_are_polynomials():
    ns, ms = inputs.radial_modes(10)
    r = np.array([1.0 + 1e-6, 1.0 - 1e-6, 1.3, -0.2])
    got = run_radial(ns, ms, r, 3)
    want = np.array(oradial.radial_table(ns, ms, r, 3))
    assert_radial_close(got, want, ns, "outside")


def test_per_mode_kernel_algorithm2():
    ns, ms = inputs.radial_modes(40)
    r = inputs.linspace_points(300)
    plan = zp.Plan(ns, ms)
    got = zp.radial_per_mode(plan, dev(r)).cpu().numpy()
    want = np.array(oradial.radial_table(ns, ms, r, 0))[0]
    assert np.max(np.abs(got - want)) < 1e-12


def test_empty_inputs_launch_nothing():
    ns, ms = inputs.radial_modes(5)
    out = zp.radial(ns, ms, dev(np.zeros(0)), 1)
    assert out.shape == (2, len(ns), 0)
    out = zp.radial([], [], dev(np.linspace(0, 1, 5)), 1)
    assert out.shape == (2, 0, 5)


def test_error_paths_leave_output_untouched():
    ns, ms = [4], [2]
    r = dev(np.linspace(0, 1, 8))
    out = torch.full((1, 1, 8), 7.0, dtype=torch.float64, device=DEV)
    lib = _lib.load()
    n = _lib.modes_i32(ns)
    m = _lib.modes_i32([3])
    st = lib.zp_radial(_lib.i32_ptr(n), _lib.i32_ptr(m), 1, r.data_ptr(), 8, 0, out.data_ptr(), None)
    assert st == 2
    host = np.zeros(8)
    st = lib.zp_radial(_lib.i32_ptr(n), _lib.i32_ptr(_lib.modes_i32(ms)), 1,
                       host.ctypes.data_as(ctypes.c_void_p), 8, 0, out.data_ptr(), None)
    assert st == 1 and b"device" in lib.zp_last_error()
    st = lib.zp_radial(_lib.i32_ptr(n), _lib.i32_ptr(_lib.modes_i32(ms)), 1, r.data_ptr() + 4, 8, 0,
                       out.data_ptr(), None)
    assert st == 1
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)
    with pytest.raises(zp.ZernikeError):
        zp.radial([5], [1], r, 4)


def test_high_order_modes_n300():
    """Modes well beyond the paper's n <= 100 (tables longer, more steps): values and all
    derivatives against the oracle, and R_n^m(1) = 1."""
    ns = [300, 300, 299, 250, 200, 300, 151]
    ms = [0, 2, 1, 250, 100, 300, 3]
    r = np.concatenate([[0.0, 1.0, 0.5], inputs.uniform_points(29, 77)[0]])
    got = run_radial(ns, ms, r, 3)
    want = np.array(oradial.radial_table(ns, ms, r, 3))
    assert_radial_close(got, want, ns, "n<=300")
    assert np.max(np.abs(got[0][:, 1] - 1.0)) < 1e-11


def test_maximum_order_modes_n1000():
    """The largest accepted order (ZP_MAX_N = 1000; 500 recursion steps for m = 0, a
    32-kilobyte table in shared memory): all derivatives against the oracle, R_n^m(1) = 1, and
    n = 1001 rejected."""
    ns = [1000, 1000, 999, 1000, 998, 1000]
    ms = [0, 1000, 1, 500, 996, 2]
    r = np.concatenate([[0.0, 1.0, 0.5, 0.999], inputs.uniform_points(12, 78)[0]])
    got = run_radial(ns, ms, r, 3)
    want = np.array(oradial.radial_table(ns, ms, r, 3))
    assert_radial_close(got, want, ns, "n=1000")
    assert np.max(np.abs(got[0][:, 1] - 1.0)) < 1e-11
    with pytest.raises(zp.ZernikeError):
        zp.radial([1001], [1], torch.as_tensor(r, device=DEV), 0)


def test_point_tables_match_direct_seeds():
    """Launches of >= 8192 points take their seeds from the per-point tables of rho^j; the
    same points in a short launch compute them directly.  Both agree with the oracle: n <= 40
    on [0, 1] with the exact endpoints, and n <= 10 at points outside [0, 1] (evaluated as
    polynomials)."""
    bulk = inputs.uniform_points(9000, 81)[0]
    for n_max, head in ((40, [0.0, 1.0, 0.5, 1e-3]), (10, [1.0 + 1e-6, 1.3, -0.2, -1.0])):
        ns, ms = inputs.radial_modes(n_max)
        r = np.concatenate([head, bulk])
        big = run_radial(ns, ms, r, 3)
        sub = np.arange(10)
        small = run_radial(ns, ms, r[sub], 3)
        want = np.array(oradial.radial_table(ns, ms, r[sub], 3))
        assert_radial_close(big[:, :, sub], want, ns, f"tables n<={n_max}")
        assert_radial_close(small, want, ns, f"direct n<={n_max}")
