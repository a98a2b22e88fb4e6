"""Parity of the tensor-core split-precision series (BF16x3 / TF32, tcgen05) with the exact oracle
and with the float64 path.

Tolerance (derived from the arithmetic): BF16x3 keeps Zh Ch + Zh Cl + Zl Ch of each product,
whose relative error is at most about 3 * 2^-16 (the dropped Zl Cl term plus the rounding of
the low halves), and the float32 accumulation adds about J * 2^-24; with Z and C first
rounded to float32 this gives |F - F64| <= 1e-4 * sum_j |Z_j C_js| + 1e-6 elementwise.  TF32
keeps 10 mantissa bits per operand (2 * 2^-11 per product): 2e-3 * sum_j |Z_j C_js| + 1e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import _lib, inputs  # noqa: E402
from oracle import basis as obasis, series as oseries  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
REL = {"bf16x3": 1e-4, "tf32": 2e-3}


def dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=DEV)


def abs_sum(ns, ms, r, th, C):
    Z = np.abs(np.array(obasis.basis_table(ns, ms, r, th, 0)[0][0]))
    return Z.T @ np.abs(C)


def wait_ok():
    assert _lib.load().zp_device_wait_status(1) == 0


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
@pytest.mark.parametrize("nmax,P,S", [(8, 128, 256), (8, 300, 5), (20, 77, 300), (3, 1, 1), (0, 5, 3)])
def test_split_small_against_oracle(prec, nmax, P, S):
    ns, ms = inputs.full_zernike_modes(nmax)
    r, th = inputs.uniform_points(P, 31 + nmax)
    C = inputs.scaled_normal_coeffs(ns, S, 31 + nmax)
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), prec).cpu().numpy()
    wait_ok()
    assert F.dtype == np.float32 and F.shape == (P, S)
    want = np.array(oseries.series_eval(ns, ms, r, th, C.tolist()))
    tol = REL[prec] * abs_sum(ns, ms, r, th, C) + 1e-6
    assert (np.abs(F - want) <= tol).all()


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_split_many_chunks_ragged_against_fp64(prec):
    """n <= 32 (561 modes: 9 K-chunks), ragged point and set tails; the full output against
    the float64 path (itself checked against the oracle) and sampled rows against the oracle."""
    ns, ms = inputs.full_zernike_modes(32)
    r, th = inputs.sqrt_uniform_points(1000, 5)
    C = inputs.scaled_normal_coeffs(ns, 300, 5)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    F = zp.series_eval(ns, ms, rt, tt, Ct, prec).double()
    wait_ok()
    F64 = zp.series_eval(ns, ms, rt, tt, Ct, "fp64")
    rel = float((F - F64).norm() / F64.norm())
    assert rel < (2e-5 if prec == "bf16x3" else 1e-3), rel
    rows = np.array([0, 127, 128, 999])
    want = np.array(oseries.series_eval(ns, ms, r[rows], th[rows], C.tolist()))
    tol = REL[prec] * abs_sum(ns, ms, r[rows], th[rows], C) + 1e-6
    assert (np.abs(F[torch.as_tensor(rows, device=DEV)].cpu().numpy() - want) <= tol).all()


def test_split_duplicates_and_scrambled_modes():
    ns = [5, 12, 12, 0, 7, 5, 30, 30]
    ms = [-3, 4, 4, 0, -7, 1, 0, -2]
    r, th = inputs.uniform_points(200, 6)
    C = inputs.scaled_normal_coeffs(np.array(ns), 40, 6)
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), "bf16x3").cpu().numpy()
    wait_ok()
    want = np.array(oseries.series_eval(ns, ms, r, th, C.tolist()))
    tol = REL["bf16x3"] * abs_sum(ns, ms, r, th, C) + 1e-6
    assert (np.abs(F - want) <= tol).all()


def test_mixed_n32_full_size_sampled():
    """The 561-mode, 1e6-point (r = sqrt(U)), 4096-set workload at full size in the
    benchmark's configuration: sampled rows against the oracle, and the relative Frobenius
    error against float64 on a 4096-point slice."""
    cfg = inputs.WORKLOADS["mixed_n32"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.sqrt_uniform_points(cfg["n_points"], cfg["seed"])
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    plan = zp.Plan(ns, ms)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    F = zp.series_eval(None, None, rt, tt, Ct, "bf16x3", plan=plan)
    torch.cuda.synchronize()
    wait_ok()
    rows = np.array([0, 1, 523_777, 999_999])
    got = F[torch.as_tensor(rows, device=DEV)].double().cpu().numpy()[:, :512]
    want = np.array(oseries.series_eval(ns, ms, r[rows], th[rows], C[:, :512].tolist()))
    tol = REL["bf16x3"] * abs_sum(ns, ms, r[rows], th[rows], C[:, :512]) + 1e-6
    assert (np.abs(got - want) <= tol).all()
    sl = slice(500_000, 504_096)
    F64 = zp.series_eval(None, None, rt[sl].contiguous(), tt[sl].contiguous(), Ct, "fp64", plan=plan)
    rel = float((F[sl].double() - F64).norm() / F64.norm())
    assert rel < 2e-5, rel
    assert bool(torch.isfinite(F).all())


@pytest.mark.parametrize("prec,code", [("bf16x3", 1), ("tf32", 2)])
@pytest.mark.parametrize("nmax,P,S", [(20, 20_000, 300), (32, 3_001, 256), (5, 129, 7)])
def test_slab_size_does_not_change_the_result(prec, code, nmax, P, S):
    """zp_series_eval (slabs of whole basis waves, ~512 MB) and zp_series_eval_static (its
    64 MB array: many smaller slabs, other CTA-pair boundaries) compute the same basis values
    and the same MMA sequence per tile, so their outputs are identical, for an odd number of
    point tiles too (a pair's missing second tile)."""
    ns, ms = inputs.full_zernike_modes(nmax)
    r, th = inputs.sqrt_uniform_points(P, 90 + nmax)
    C = inputs.scaled_normal_coeffs(ns, S, 90 + nmax)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    regular = zp.series_eval(ns, ms, rt, tt, Ct, prec)
    lib = _lib.load()
    n, m = _lib.modes_i32(ns), _lib.modes_i32(ms)
    static = torch.full((P, S), float("nan"), dtype=torch.float32, device=DEV)
    _lib.check("zp_series_eval_static", lib.zp_series_eval_static(
        _lib.i32_ptr(n), _lib.i32_ptr(m), len(n), rt.data_ptr(), tt.data_ptr(), P, Ct.data_ptr(), S, code,
        static.data_ptr(), torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    wait_ok()
    assert torch.equal(regular, static)


def test_split_long_column_plan():
    """Modes of order 900 and 899 (451-step columns) beside a small full set, against the
    float64 path."""
    ns, ms = inputs.full_zernike_modes(6)
    ns = list(ns) + [900, 899]
    ms = list(ms) + [0, -1]
    r, th = inputs.sqrt_uniform_points(700, 95)
    C = inputs.scaled_normal_coeffs(np.asarray(ns), 40, 95)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    for prec in ("bf16x3", "tf32"):
        F = zp.series_eval(ns, ms, rt, tt, Ct, prec).double()
        F64 = zp.series_eval(ns, ms, rt, tt, Ct, "fp64")
        z = zp.basis(ns, ms, rt, tt, 0)[0][0].abs()
        bound = REL[prec] * (z.T @ Ct.abs()) + 1e-6
        wait_ok()
        assert bool(((F - F64).abs() <= bound).all())


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_split_step_descriptors_irregular_and_odd_steps(prec):
    """Recursion steps of every slot shape the basis kernel's per-step descriptors take: one
    slot, odd counts with mixed cos/sin flags, exactly 24 slots (the most a descriptor's flags
    hold), and 26 and 40 slots (beyond them: the slots are read one by one), in caller order
    with duplicates; against the oracle."""
    ns, ms = [], []
    ns += [10, 10] * 13                  # one step with 26 slots (alternating cos / sin)
    ms += [2, -2] * 13
    ns += [7] * 24                       # exactly 24 slots, mixed flags
    ms += [3, -3, -3, 3, 3, 3, -3, -3] * 3
    ns += [6, 6, 6]                      # three cos slots (odd count)
    ms += [0, 0, 0]
    ns += [8, 8, 8]                      # odd count, mixed flags
    ms += [4, -4, -4]
    ns += [12] * 40                      # 40 sin slots
    ms += [-6] * 40
    ns += [5, 3, 1, 9, 0, 11]            # single-slot steps in other columns
    ms += [1, -1, 1, -9, 0, 11]
    order = np.random.default_rng(5).permutation(len(ns))
    ns = [ns[i] for i in order]
    ms = [ms[i] for i in order]
    r, th = inputs.uniform_points(150, 44)
    C = inputs.scaled_normal_coeffs(ns, 37, 44)
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), prec).cpu().numpy()
    wait_ok()
    want = np.array(oseries.series_eval(ns, ms, r, th, C.tolist()))
    tol = REL[prec] * abs_sum(ns, ms, r, th, C) + 1e-6
    assert (np.abs(F - want) <= tol).all()


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "fp64emu"])
@pytest.mark.parametrize("nmax,P,S", [(32, 3_001, 300), (20, 129, 256), (8, 20_000, 17)])
def test_cta_pairs_match_single_ctas(prec, nmax, P, S, monkeypatch):
    """The GEMM on CTA pairs (256-point tiles, cta_group::2 MMAs, half of B in each CTA) and on
    single CTAs (ZP_GEMM_CTA_PAIRS=0, read at every launch) run the same MMA sequence for every
    output: identical results, for odd point-tile counts too (a pair's missing second tile)."""
    ns, ms = inputs.full_zernike_modes(nmax)
    r, th = inputs.sqrt_uniform_points(P, 140 + nmax)
    C = inputs.scaled_normal_coeffs(ns, S, 140 + nmax)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    paired = zp.series_eval(ns, ms, rt, tt, Ct, prec)
    torch.cuda.synchronize()
    wait_ok()
    monkeypatch.setenv("ZP_GEMM_CTA_PAIRS", "0")
    single = zp.series_eval(ns, ms, rt, tt, Ct, prec)
    torch.cuda.synchronize()
    wait_ok()
    assert torch.equal(paired, single)
