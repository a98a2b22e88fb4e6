"""The fused float64-accurate series for up to 16 coefficient sets (zp_series_eval with
ZP_PREC_FP64_EMULATED routes there): the basis is generated inside the tensor-core kernel.
Checked against the exact oracle at the float64 tolerance, against the unfused emulated path
and the DGEMM baseline at larger sizes, on ragged tiles, scrambled and duplicated mode lists,
points off the unit disc (the kernel's first pass over the point's modes), non-finite inputs,
the 5041-mode limit, and in the batched forward (graph capture, determinism, full size)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import _lib, inputs  # noqa: E402
from oracle import basis as obasis, series as oseries  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=DEV)


def abs_bound(ns, ms, r, th, C):
    Z = np.abs(np.array(obasis.basis_table(ns, ms, r, th, 0)[0][0]))
    return Z.T @ np.abs(C)


def check_waits():
    torch.cuda.synchronize()
    assert _lib.load().zp_device_wait_status(1) == 0


@pytest.mark.parametrize("nmax,P,S", [(8, 300, 5), (3, 1, 1), (12, 129, 16), (0, 4, 2), (20, 127, 7), (6, 257, 16)])
def test_fused_against_oracle(nmax, P, S):
    ns, ms = inputs.full_zernike_modes(nmax)
    r, th = inputs.uniform_points(P, 70 + nmax)
    if P > 3:
        r[:3] = [0.0, 1.0, 1e-3]  # the origin, the unit circle, a point where high powers underflow
    C = inputs.scaled_normal_coeffs(ns, S, 70 + nmax) * 11.0
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), "fp64emu").cpu().numpy()
    check_waits()
    want = np.array(oseries.series_eval(ns, ms, r, th, C.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r, th, C))
    assert (np.abs(F - want) <= tol).all(), float(np.max(np.abs(F - want) / tol))


def test_fused_scrambled_duplicated_modes():
    ns = [40, 3, 3, 0, 17, 40, 22, 9, 2, 2, 31]
    ms = [-2, 1, 1, 0, -17, 38, 0, -9, -2, 2, 31]
    r, th = inputs.sqrt_uniform_points(1000, 5)
    C = np.random.default_rng(5).standard_normal((len(ns), 9))
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), "fp64emu").cpu().numpy()
    check_waits()
    rows = np.array([0, 1, 127, 128, 500, 999])
    want = np.array(oseries.series_eval(ns, ms, r[rows], th[rows], C.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r[rows], th[rows], C))
    assert (np.abs(F[rows] - want) <= tol).all()
    # Duplicated modes give identical columns' contributions: doubling a coefficient of one copy
    # equals moving it to the other.
    C2 = C.copy()
    C2[1] += C2[2]
    C2[2] = 0.0
    F2 = zp.series_eval(ns, ms, dev(r), dev(th), dev(C2), "fp64emu").cpu().numpy()
    assert np.max(np.abs(F2 - F)) <= 1e-13 * (1.0 + np.max(np.abs(F)))


def test_fused_points_off_the_disc_and_non_finite():
    """r outside [0, 1] takes the per-point first pass for its scale; NaN points give NaN rows and
    a set holding an infinity or a NaN gives a NaN column, every other output float64-exact."""
    ns, ms = inputs.full_zernike_modes(10)
    r, th = inputs.uniform_points(300, 9)
    r[10:20] = np.linspace(1.0, 1.4, 10)
    r[20:25] = -np.linspace(0.1, 0.9, 5)
    r[7] = np.nan
    th[8] = np.inf
    th[9] = np.nan
    th[30] = 1e300  # finite: evaluated, by angle addition from cos/sin(theta)
    C = inputs.scaled_normal_coeffs(ns, 6, 9)
    C[4, 1] = np.inf
    F = zp.series_eval(ns, ms, dev(r), dev(th), dev(C), "fp64emu").cpu().numpy()
    check_waits()
    assert np.isnan(F[7]).all() and np.isnan(F[8]).all() and np.isnan(F[9]).all() and np.isnan(F[:, 1]).all()
    assert np.isfinite(F[30, [0, 2, 3, 4, 5]]).all()
    ok_rows = np.array([p for p in range(300) if p not in (7, 8, 9, 30)])
    cols = [0, 2, 3, 4, 5]
    Cg = C[:, cols]
    want = np.array(oseries.series_eval(ns, ms, r[ok_rows], th[ok_rows], Cg.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r[ok_rows], th[ok_rows], Cg))
    got = F[np.ix_(ok_rows, cols)]
    assert (np.abs(got - want) <= tol).all(), float(np.max(np.abs(got - want) / tol))


def test_fused_against_unfused_and_dgemm_at_the_mode_limit():
    """4950 modes (full set n <= 98, under the 5041-mode limit of exact float32 diagonal sums):
    the fused result against the DGEMM baseline; 16 sets fused against 17 sets unfused (the
    same first 16 columns)."""
    ns, ms = inputs.full_zernike_modes(98)
    r, th = inputs.sqrt_uniform_points(3000, 13)
    C = inputs.scaled_normal_coeffs(ns, 17, 13)
    rt, tt = dev(r), dev(th)
    plan = zp.Plan(ns, ms)
    F16 = zp.series_eval(None, None, rt, tt, dev(C[:, :16]), "fp64emu", plan=plan)
    F17 = zp.series_eval(None, None, rt, tt, dev(C), "fp64emu", plan=plan)
    Fd = zp.series_eval(None, None, rt, tt, dev(C[:, :16]), "fp64", plan=plan)
    check_waits()
    Z = zp.basis(None, None, rt, tt, 0, plan=plan)[0][0].abs()
    bound = 1e-13 * (1.0 + Z.T @ dev(np.abs(C[:, :16])))
    assert bool(((F16 - Fd).abs() <= bound).all())
    assert bool(((F16 - F17[:, :16]).abs() <= bound).all())
    # one more mode than the limit goes to the unfused path and still agrees
    ns2, ms2 = list(ns) + [99] * 92, list(ms) + list(range(-99, 85, 2))
    assert len(ns2) == 5042
    C2 = np.random.default_rng(2).standard_normal((5042, 4)) * 0.01
    rows = slice(0, 256)
    Fa = zp.series_eval(ns2, ms2, rt[rows].contiguous(), tt[rows].contiguous(), dev(C2), "fp64emu")
    Fb = zp.series_eval(ns2, ms2, rt[rows].contiguous(), tt[rows].contiguous(), dev(C2), "fp64")
    check_waits()
    assert float((Fa - Fb).abs().max()) <= 1e-12 * (1.0 + float(Fb.abs().max()))


def test_fused_series_n24_points_full_size_sampled():
    """The 325-mode, 50000-point polar grid with 16 sets, sampled rows against the oracle, and
    two calls bit for bit equal (deterministic)."""
    cfg = inputs.WORKLOADS["series_n24"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.polar_grid(cfg["n_r"], cfg["n_theta"])
    C = inputs.scaled_normal_coeffs(ns, 16, cfg["seed"])
    plan = zp.Plan(ns, ms)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    F = zp.series_eval(None, None, rt, tt, Ct, "fp64emu", plan=plan)
    F2 = zp.series_eval(None, None, rt, tt, Ct, "fp64emu", plan=plan)
    check_waits()
    assert torch.equal(F, F2)
    rows = np.array([0, 1, 199, 200, 24_999, 49_999, 31_337])
    want = np.array(oseries.series_eval(ns, ms, r[rows], th[rows], C.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(ns, ms, r[rows], th[rows], C))
    assert (np.abs(F[torch.as_tensor(rows, device=DEV)].cpu().numpy() - want) <= tol).all()


def make_instances(specs, S, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k, (n_max, P) in enumerate(specs):
        ns, ms = inputs.full_zernike_modes(n_max)
        r, th = inputs.uniform_points(P, seed * 100 + k)
        C = rng.standard_normal((len(ns), S))
        out.append({"n": ns, "m": ms, "r": dev(r), "theta": dev(th), "coeffs": dev(C), "_r": r, "_th": th, "_C": C})
    return out


@pytest.mark.parametrize("S", [3, 16])
def test_batched_fused_forward_matches_oracle_and_dfma_path(S):
    specs = [(20, 777), (0, 5), (3, 1), (8, 300), (15, 100), (1, 64), (20, 129), (12, 0), (6, 33), (40, 1000)]
    inst = make_instances(specs, S, seed=S)
    b = zp.Batch(inst, S, with_adjoint=False)
    b.forward("fp64emu")
    torch.cuda.synchronize()
    got = [rec["out"].clone() for rec in b.instances]
    b.forward("fp64")
    check_waits()
    for d, g, rec in zip(inst, got, b.instances):
        if len(d["_r"]) == 0:
            continue
        assert float((g - rec["out"]).abs().max()) <= 1e-12 * (1.0 + float(rec["out"].abs().max()))
    for i, rows in ((0, [0, 1, 776]), (9, [0, 127, 128, 999]), (2, [0])):
        d = inst[i]
        want = np.array(oseries.series_eval(d["n"], d["m"], d["_r"][rows], d["_th"][rows], d["_C"].tolist()))
        tol = 1e-13 * (1.0 + abs_bound(d["n"], d["m"], d["_r"][rows], d["_th"][rows], d["_C"]))
        assert (np.abs(got[i][rows].cpu().numpy() - want) <= tol).all()


def test_batched_fused_forward_graph_capture_and_determinism():
    inst = make_instances([(30, 2000), (7, 130), (50, 400)], 16, seed=21)
    b = zp.Batch(inst, 16, with_adjoint=False)
    b.forward("fp64emu")
    torch.cuda.synchronize()
    first = [rec["out"].clone() for rec in b.instances]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for rec in b.instances:
            rec["out"].zero_()
        with torch.cuda.graph(g, stream=s):
            b.forward("fp64emu")
    torch.cuda.current_stream().wait_stream(s)
    for rec in b.instances:
        rec["out"].fill_(7.0)
    g.replay()
    check_waits()
    for a, rec in zip(first, b.instances):
        assert torch.equal(a, rec["out"])
    # New coefficient values in place: the captured graph re-cuts them on replay.  Doubling
    # every coefficient raises each set's scale by one and leaves its digits unchanged, so the
    # result doubles exactly (a sign change would not: the balanced digits of -X are not always
    # the negated digits of X, and the dropped low-order pairs then differ).
    for d in inst:
        d["coeffs"].mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    for a, rec in zip(first, b.instances):
        assert torch.equal(2.0 * a, rec["out"])


def test_batched_512_fused_full_size_sampled():
    """512 instances, n_max ~ U{8..64}, points log-uniform in [1e3, 2e5], 16 sets: the fused
    float64-accurate forward, sampled instances against the single-instance DGEMM baseline and
    one instance's rows against the oracle."""
    cfg = inputs.WORKLOADS["batched_512"]
    raw = inputs.batched_instances(cfg["n_instances"], cfg["n_sets"], cfg["seed"])
    inst = [{"n": x.n, "m": x.m, "r": dev(x.r), "theta": dev(x.theta), "coeffs": dev(x.coeffs)} for x in raw]
    b = zp.Batch(inst, cfg["n_sets"], with_adjoint=False)
    b.forward("fp64emu")
    check_waits()
    for i in (0, 17, 255, 511):
        d, rec = inst[i], b.instances[i]
        want = zp.series_eval(d["n"], d["m"], d["r"], d["theta"], d["coeffs"], "fp64")
        assert float((rec["out"] - want).abs().max()) <= 1e-12 * (1 + float(want.abs().max()))
    x = raw[17]
    rows = [0, len(x.r) - 1]
    want = np.array(oseries.series_eval(x.n, x.m, x.r[rows], x.theta[rows], x.coeffs.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(x.n, x.m, x.r[rows], x.theta[rows], x.coeffs))
    assert (np.abs(b.instances[17]["out"][rows].cpu().numpy() - want) <= tol).all()


@pytest.mark.parametrize("nmax", [49, 50])
def test_fused_on_both_sides_of_the_short_digit_shape(nmax):
    """n <= 49 (1472 padded positions) takes 9 digits of 6 bits, n <= 50 (1504) 11 digits of 5
    bits: both against the DGEMM baseline within the float64 bound, forward and the adjoint's
    fused point gradients, with coefficients that fill the digit range."""
    ns, ms = inputs.full_zernike_modes(nmax)
    r, th = inputs.sqrt_uniform_points(2000, 60 + nmax)
    r[:3] = [1.0, 0.999, 0.0]
    C = np.random.default_rng(nmax).standard_normal((len(ns), 16))
    rt, tt, Ct = dev(r), dev(th), dev(C)
    plan = zp.Plan(ns, ms)
    F = zp.series_eval(None, None, rt, tt, Ct, "fp64emu", plan=plan)
    Fd = zp.series_eval(None, None, rt, tt, Ct, "fp64", plan=plan)
    check_waits()
    Z = zp.basis(None, None, rt, tt, 0, plan=plan)[0][0].abs()
    bound = 1e-13 * (1.0 + Z.T @ Ct.abs())
    assert bool(((F - Fd).abs() <= bound).all())
    G = dev(np.random.default_rng(nmax + 1).standard_normal((len(r), 16)))
    _, gr, gt = zp.series_adjoint(None, None, rt, tt, Ct, G, need=(False, True, True), plan=plan, prec="fp64emu")
    _, wr, wt = zp.series_adjoint(None, None, rt, tt, Ct, G, need=(False, True, True), plan=plan, prec="fp64")
    check_waits()
    # |dZ_j/drho| <= n_j^2 (Markov) and |dZ_j/dtheta| <= |m_j| <= n_j on the disc: per point,
    # sum_s |G[p][s]| sum_j n_j^2 |C[j][s]| bounds the terms either gradient sums
    w = dev((np.asarray(ns, dtype=np.float64) ** 2)[:, None] * np.abs(C)).sum(0)
    scale = 1.0 + G.abs() @ w
    assert bool(((gr - wr).abs() <= 1e-13 * scale).all())
    assert bool(((gt - wt).abs() <= 1e-13 * scale).all())
