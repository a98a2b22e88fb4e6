"""The allocation-free series entry point, zp_series_eval_static.

Callers that cannot allocate device memory while they run (host callbacks, allocator hooks,
applications that reserve all device memory up front) use this entry point: its scratch is a
fixed device array inside the library.  These tests call it through the C ABI and compare
its output with the ordinary zp_series_eval on the same inputs, twice in a row with
different problems (the shared array must be fully rewritten by each call), and check that
a problem too large for the array is refused before anything runs.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import _lib, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PREC_CODE = {"bf16x3": 1, "tf32": 2}
REL = {"bf16x3": 1e-4, "tf32": 2e-3}  # the split-precision tolerances of the other series tests


def dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=DEV)


def call_static(ns, ms, r, th, C, prec):
    lib = _lib.load()
    n, m = _lib.modes_i32(ns), _lib.modes_i32(ms)
    out = torch.full((r.numel(), C.shape[1]), float("nan"), dtype=torch.float32, device=DEV)
    st = lib.zp_series_eval_static(_lib.i32_ptr(n), _lib.i32_ptr(m), len(n), r.data_ptr(), th.data_ptr(), r.numel(),
                                   C.data_ptr(), C.shape[1], PREC_CODE[prec], out.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    _lib.check("zp_series_eval_static", st)
    return out


def compare(ns, ms, P, S, prec, seed):
    """The static entry point runs the same split kernels on the same inputs as zp_series_eval
    (only the scratch differs), so the two agree bit for bit; a stale tile or a wrong slab offset
    in the shared array would break that."""
    r, th = inputs.sqrt_uniform_points(P, seed)
    C = inputs.scaled_normal_coeffs(np.asarray(ns), S, seed)
    rt, tt, Ct = dev(r), dev(th), dev(C)
    got = call_static(ns, ms, rt, tt, Ct, prec)
    want = zp.series_eval(ns, ms, rt, tt, Ct, prec)
    torch.cuda.synchronize()
    assert _lib.load().zp_device_wait_status(1) == 0
    assert bool(torch.isfinite(got).all())
    assert torch.equal(got, want), float((got.double() - want.double()).abs().max())
    return r, th, C, got


def test_static_matches_series_eval_twice_in_a_row():
    # First call: 561 modes and 60000 points, several slabs of the static array.
    ns, ms = inputs.full_zernike_modes(32)
    compare(ns, ms, 60_000, 512, "bf16x3", 41)
    # Second call: a smaller, different (scrambled, duplicated) mode list, fewer sets, ragged
    # sizes, TF32: every byte it reads must come from this call, not from the first.
    ns2 = [40, 3, 3, 0, 17, 40, 22, 9]
    ms2 = [-2, 1, 1, 0, -17, 38, 0, -9]
    compare(ns2, ms2, 1_001, 37, "tf32", 42)
    # Third call: the small problem again in BF16x3, checked against the exact oracle too.
    from oracle import series as oseries

    r, th, C, got = compare(ns2, ms2, 40, 5, "bf16x3", 43)
    want = np.array(oseries.series_eval(ns2, ms2, r, th, C.tolist()))
    z = zp.basis(ns2, ms2, dev(r), dev(th), 0)[0][0].abs().cpu().numpy()
    bound = REL["bf16x3"] * (z.T @ np.abs(C)) + 1e-6
    assert (np.abs(got.double().cpu().numpy() - want) <= bound).all()


def test_static_refuses_stream_capture():
    ns, ms = inputs.full_zernike_modes(4)
    r, th = inputs.uniform_points(64, 3)
    rt, tt = dev(r), dev(th)
    C = torch.ones((len(ns), 8), dtype=torch.float64, device=DEV)
    out = torch.full((64, 8), 5.0, dtype=torch.float32, device=DEV)
    lib = _lib.load()
    n, m = _lib.modes_i32(ns), _lib.modes_i32(ms)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            st = lib.zp_series_eval_static(_lib.i32_ptr(n), _lib.i32_ptr(m), len(n), rt.data_ptr(), tt.data_ptr(), 64,
                                           C.data_ptr(), 8, 1, out.data_ptr(), side.cuda_stream)
    assert st == 1  # ZP_ERR_INVALID_ARG
    assert b"captured" in lib.zp_last_error()
    torch.cuda.synchronize()
    assert bool((out == 5.0).all())


def test_static_rejects_problems_beyond_its_array():
    ns, ms = inputs.full_zernike_modes(200)  # 20301 modes
    r, th = inputs.uniform_points(10, 1)
    C = torch.zeros((len(ns), 4096), dtype=torch.float64, device=DEV)
    lib = _lib.load()
    n, m = _lib.modes_i32(ns), _lib.modes_i32(ms)
    out = torch.full((10, 4096), 3.0, dtype=torch.float32, device=DEV)
    rt, tt = dev(r), dev(th)
    st = lib.zp_series_eval_static(_lib.i32_ptr(n), _lib.i32_ptr(m), len(n), rt.data_ptr(), tt.data_ptr(), 10,
                                   C.data_ptr(), 4096, 1, out.data_ptr(), None)
    assert st == 1  # ZP_ERR_INVALID_ARG
    assert b"ZP_STATIC_SCRATCH_BYTES" in lib.zp_last_error()
    torch.cuda.synchronize()
    assert bool((out == 3.0).all())
    st = lib.zp_series_eval_static(_lib.i32_ptr(n), _lib.i32_ptr(m), len(n), rt.data_ptr(), tt.data_ptr(), 10,
                                   C.data_ptr(), 4096, 0, out.data_ptr(), None)
    assert st == 1  # float64 is not offered here
    # A set count so large that the tile sizes would wrap around in 64-bit arithmetic.
    few_n, few_m = _lib.modes_i32([0, 1]), _lib.modes_i32([0, 1])
    for huge in (1 << 40, (1 << 62) // 3):
        st = lib.zp_series_eval_static(_lib.i32_ptr(few_n), _lib.i32_ptr(few_m), 2, rt.data_ptr(), tt.data_ptr(), 10,
                                       C.data_ptr(), huge, 1, out.data_ptr(), None)
        assert st == 1
    torch.cuda.synchronize()
    assert bool((out == 3.0).all())
