"""Batched uneven series (zp_batch_*): parity with the oracle and with the single-instance
entry points, determinism, CUDA-graph capture and the autotuner."""
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


def make_instances(specs, S, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k, (n_max, P) in enumerate(specs):
        ns, ms = inputs.full_zernike_modes(n_max)
        r, th = inputs.uniform_points(P, seed * 100 + k)
        C = rng.standard_normal((len(ns), S))
        G = rng.standard_normal((P, S))
        out.append({"n": ns, "m": ms, "r": dev(r), "theta": dev(th), "coeffs": dev(C), "grad_out": dev(G),
                    "_r": r, "_th": th, "_C": C, "_G": G})
    return out


SPECS = [(20, 777), (0, 5), (3, 1), (8, 300), (15, 100), (1, 64), (20, 129), (12, 0), (6, 33)]


def abs_bound(ns, ms, r, th, C):
    Z = np.abs(np.array(obasis.basis_table(ns, ms, r, th, 0)[0][0]))
    return Z.T @ np.abs(C)


@pytest.mark.parametrize("S", [5, 20])
def test_batched_forward_matches_oracle_and_single_path(S):
    inst = make_instances(SPECS, S, seed=S)
    b = zp.Batch(inst, S)
    b.forward("fp64")
    torch.cuda.synchronize()
    for d, rec in zip(inst, b.instances):
        if len(d["_r"]) == 0:
            continue
        got = rec["out"]
        want = zp.series_eval(d["n"], d["m"], d["r"], d["theta"], d["coeffs"])
        scale = 1e-12 * (1.0 + float(want.abs().max()))
        assert float((got - want).abs().max()) <= scale
    # oracle on a few rows of the biggest instance
    d, rec = inst[0], b.instances[0]
    rows = [0, 1, 776]
    want = np.array(oseries.series_eval(d["n"], d["m"], d["_r"][rows], d["_th"][rows], d["_C"].tolist()))
    tol = 1e-13 * (1.0 + abs_bound(d["n"], d["m"], d["_r"][rows], d["_th"][rows], d["_C"]))
    assert (np.abs(rec["out"][rows].cpu().numpy() - want) <= tol).all()


def test_batched_forward_fp32():
    S = 16
    inst = make_instances(SPECS, S, seed=3)
    b64 = zp.Batch(inst, S)
    b32 = zp.Batch(inst, S, out_dtype=torch.float32, with_adjoint=False)
    b64.forward("fp64")
    b32.forward("fp32")
    torch.cuda.synchronize()
    for r64, r32 in zip(b64.instances, b32.instances):
        if r64["out"].numel() == 0:
            continue
        rel = float((r32["out"].double() - r64["out"]).norm() / r64["out"].norm())
        assert rel < 2e-6, rel


@pytest.mark.parametrize("prec", ["fp64", "fp64emu"])
@pytest.mark.parametrize("S", [5, 20])
def test_batched_adjoint_matches_single_path_and_is_deterministic(S, prec):
    """Both contractions against the single-series adjoint (for "fp64emu" grad_coeffs comes from
    the same tensor-core kernels per instance: identical), and a second run bitwise equal to
    the first."""
    inst = make_instances(SPECS, S, seed=10 + S)
    b = zp.Batch(inst, S)
    b.adjoint(prec)
    torch.cuda.synchronize()
    first = [tuple(rec[k].clone() for k in ("grad_coeffs", "grad_r", "grad_theta")) for rec in b.instances]
    for d, rec in zip(inst, b.instances):
        gC, gr, gt = zp.series_adjoint(d["n"], d["m"], d["r"], d["theta"], d["coeffs"], d["grad_out"])
        for got, want in ((rec["grad_coeffs"], gC), (rec["grad_r"], gr), (rec["grad_theta"], gt)):
            if want.numel() == 0:
                continue
            if prec == "fp64emu" and got is rec["grad_coeffs"]:
                assert torch.equal(got, want)
            scale = 1e-11 * (1.0 + float(want.abs().max()))
            assert float((got - want).abs().max()) <= scale
    b.adjoint(prec)
    torch.cuda.synchronize()
    for f, rec in zip(first, b.instances):
        for a, k in zip(f, ("grad_coeffs", "grad_r", "grad_theta")):
            assert torch.equal(a, rec[k]), k  # bitwise identical (two-addend atomic sums are order-free)


@pytest.mark.parametrize("prec", ["fp64", "fp64emu"])
def test_batched_adjoint_against_oracle_small(prec):
    S = 3
    inst = make_instances([(5, 40), (2, 7)], S, seed=7)
    b = zp.Batch(inst, S)
    b.adjoint(prec)
    torch.cuda.synchronize()
    for d, rec in zip(inst, b.instances):
        wC, wr, wt = oseries.series_adjoint(d["n"], d["m"], d["_r"], d["_th"], d["_C"].tolist(), d["_G"].tolist())
        assert np.max(np.abs(rec["grad_coeffs"].cpu().numpy() - np.array(wC))) < 1e-12
        assert np.max(np.abs(rec["grad_r"].cpu().numpy() - np.array(wr))) < 1e-11
        assert np.max(np.abs(rec["grad_theta"].cpu().numpy() - np.array(wt))) < 1e-11


def test_batched_emulated_adjoint_off_disc_points():
    """Points beyond the unit disc (r up to 1.4) take the fused kernel's per-point row scale for
    the derivative series too: grad_r and grad_theta against the float64 CUDA-core form."""
    S = 16
    inst = make_instances([(20, 500), (9, 77), (0, 30)], S, seed=41)
    rng = np.random.default_rng(5)
    for d in inst:
        r = rng.uniform(0.0, 1.4, len(d["_r"]))
        d["_r"] = r
        d["r"] = dev(r)
    b = zp.Batch(inst, S)
    b.adjoint("fp64")
    torch.cuda.synchronize()
    ref = [tuple(rec[k].clone() for k in ("grad_coeffs", "grad_r", "grad_theta")) for rec in b.instances]
    b.adjoint("fp64emu")
    torch.cuda.synchronize()
    for f, rec in zip(ref, b.instances):
        for want, k in zip(f, ("grad_coeffs", "grad_r", "grad_theta")):
            if want.numel() == 0:
                continue
            got = rec[k]
            assert bool(torch.isfinite(got).all())
            scale = 1e-11 * (1.0 + float(want.abs().max()))
            assert float((got - want).abs().max()) <= scale, k


def test_batched_cuda_graph_and_tuner():
    S = 16
    inst = make_instances(SPECS, S, seed=21)
    b = zp.Batch(inst, S)
    b.forward("fp64")
    torch.cuda.synchronize()
    ref = [rec["out"].clone() for rec in b.instances]
    cfg, best = b.tune("forward", "fp64", reps=1)
    assert best > 0 and cfg[0] in (64, 128, 256)
    assert b.config() == cfg
    for rec in b.instances:
        rec["out"].zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.forward("fp64")
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    for a, rec in zip(ref, b.instances):
        assert torch.equal(a, rec["out"])
    cfg2, _ = b.tune("adjoint", reps=1)
    b.adjoint("fp64")
    torch.cuda.synchronize()
    d, rec = inst[0], b.instances[0]
    gC, gr, gt = zp.series_adjoint(d["n"], d["m"], d["r"], d["theta"], d["coeffs"], d["grad_out"])
    assert float((rec["grad_coeffs"] - gC).abs().max()) <= 1e-11 * (1 + float(gC.abs().max()))


def test_batched_512_full_size_sampled():
    """512 instances, n_max ~ U{8..64}, points log-uniform in [1e3, 2e5], 16 sets: the full
    batch forward in float64, sampled instances against the single-instance path; the
    per-instance launch variant gives identical results."""
    cfg = inputs.WORKLOADS["batched_512"]
    raw = inputs.batched_instances(cfg["n_instances"], cfg["n_sets"], cfg["seed"])
    inst = [{"n": x.n, "m": x.m, "r": dev(x.r), "theta": dev(x.theta), "coeffs": dev(x.coeffs)} for x in raw]
    b = zp.Batch(inst, cfg["n_sets"], with_adjoint=False)
    b.forward("fp64")
    torch.cuda.synchronize()
    for i in (0, 17, 255, 511):
        d, rec = inst[i], b.instances[i]
        want = zp.series_eval(d["n"], d["m"], d["r"], d["theta"], d["coeffs"])
        assert float((rec["out"] - want).abs().max()) <= 1e-12 * (1 + float(want.abs().max()))
    # one instance's rows directly against the oracle
    x = raw[17]
    rows = [0, len(x.r) - 1]
    want = np.array(oseries.series_eval(x.n, x.m, x.r[rows], x.theta[rows], x.coeffs.tolist()))
    tol = 1e-13 * (1.0 + abs_bound(x.n, x.m, x.r[rows], x.theta[rows], x.coeffs))
    assert (np.abs(b.instances[17]["out"][rows].cpu().numpy() - want) <= tol).all()
    keep = [rec["out"].clone() for rec in b.instances[:8]]
    b.forward_per_instance()
    torch.cuda.synchronize()
    for a, rec in zip(keep, b.instances[:8]):
        assert torch.equal(a, rec["out"])


def test_batched_512_full_size_adjoint_emulated_against_float64():
    """The full batched_512 adjoint: the float64-accurate form (two fused derivative-series
    passes, per-instance tensor-core grad_C) against the float64 CUDA-core form on every
    instance, and one instance's point gradients against the oracle."""
    cfg = inputs.WORKLOADS["batched_512"]
    raw = inputs.batched_instances(cfg["n_instances"], cfg["n_sets"], cfg["seed"])
    rng = np.random.default_rng(77)
    inst = [{"n": x.n, "m": x.m, "r": dev(x.r), "theta": dev(x.theta), "coeffs": dev(x.coeffs),
             "grad_out": dev(rng.standard_normal((len(x.r), cfg["n_sets"])))} for x in raw]
    b = zp.Batch(inst, cfg["n_sets"])
    b.adjoint("fp64")
    torch.cuda.synchronize()
    ref = [tuple(rec[k].clone() for k in ("grad_coeffs", "grad_r", "grad_theta")) for rec in b.instances]
    b.adjoint("fp64emu")
    torch.cuda.synchronize()
    for f, rec in zip(ref, b.instances):
        for want, k in zip(f, ("grad_coeffs", "grad_r", "grad_theta")):
            if want.numel() == 0:
                continue
            got = rec[k]
            assert float((got - want).abs().max()) <= 1e-11 * (1.0 + float(want.abs().max())), k
    x, rec = raw[17], b.instances[17]
    rows = [0, len(x.r) - 1]
    G = inst[17]["grad_out"][rows].cpu().numpy()
    _, wr, wt = oseries.series_adjoint(x.n, x.m, x.r[rows], x.theta[rows], x.coeffs.tolist(), G.tolist())
    scale = 1.0 + np.abs(G).sum(1) * np.abs(x.coeffs).sum() * max(x.n) ** 2
    assert (np.abs(rec["grad_r"][rows].cpu().numpy() - np.array(wr)) <= 1e-12 * scale).all()
    assert (np.abs(rec["grad_theta"][rows].cpu().numpy() - np.array(wt)) <= 1e-12 * scale).all()
    b.close()
