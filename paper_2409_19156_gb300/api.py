"""Python front end: torch tensors in, torch tensors out, every step in the CUDA library.

Functions mirror the C ABI (include/zernike_gb300.h):
    radial(n, m, r, max_deriv)            -> [K][J][P] float64
    basis(n, m, r, theta, max_deriv)      -> ([K][J][P], dtheta [J][P] or None)
    radial_per_mode(plan, r)              -> [J][P] (Algorithm 2 comparison kernel)
    series_eval(n, m, r, theta, C, prec)  -> [P][S] (float64, or float32 for split precision)
    series_adjoint(n, m, r, theta, C, G)  -> (grad_C, grad_r, grad_theta)
`n`, `m` are host integer sequences; r, theta, C, G are CUDA float64 tensors.  Work is
enqueued on torch's current stream of the tensors' device.

Precisions: "fp64emu" (the default for float64 results: contractions on the library's
float64-accurate tensor-core GEMM), "fp64" (the plain basis-then-cuBLAS-DGEMM baseline),
"bf16x3" and "tf32" (split-precision tensor-core contraction, float32 results).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

PREC = {"fp64": 0, "bf16x3": 1, "tf32": 2, "fp64emu": 4}


def _stream(device: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_f64(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    return t.contiguous()


class Plan:
    """A mode list prepared once (validated, grouped by |m|, tables on the device)."""

    def __init__(self, n, m, device=None):
        self.n = _lib.modes_i32(n)
        self.m = _lib.modes_i32(m)
        if self.n.shape != self.m.shape or self.n.ndim != 1:
            raise ValueError("n and m must be 1-D sequences of equal length")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        handle = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _lib.call("zp_plan_create", _lib.i32_ptr(self.n), _lib.i32_ptr(self.m), len(self.n), ctypes.byref(handle))
        self.handle = handle

    @property
    def n_modes(self) -> int:
        return len(self.n)

    def info(self) -> dict:
        nm, nmax, ncol = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _lib.call("zp_plan_info", self.handle, ctypes.byref(nm), ctypes.byref(nmax), ctypes.byref(ncol))
        return {"n_modes": nm.value, "n_max": nmax.value, "n_columns": ncol.value}

    def close(self):
        if getattr(self, "handle", None):
            _lib.call("zp_plan_destroy", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def radial(n, m, r: torch.Tensor, max_deriv: int = 0, plan: Plan | None = None, out=None) -> torch.Tensor:
    r = _dev_f64(r, "r")
    nn, mm = (plan.n, plan.m) if plan is not None else (_lib.modes_i32(n), _lib.modes_i32(m))
    J, P = len(nn), r.numel()
    if out is None:
        out = torch.empty((max_deriv + 1, J, P), dtype=torch.float64, device=r.device)
    st = _stream(r.device)
    with torch.cuda.device(r.device):
        if plan is not None:
            _lib.call("zp_radial_plan", plan.handle, r.data_ptr(), P, max_deriv, out.data_ptr(), st)
        else:
            _lib.call("zp_radial", _lib.i32_ptr(nn), _lib.i32_ptr(mm), J, r.data_ptr(), P, max_deriv,
                      out.data_ptr(), st)
    return out


def basis(n, m, r: torch.Tensor, theta: torch.Tensor, max_deriv: int = 0, dtheta: bool = False,
          plan: Plan | None = None):
    r = _dev_f64(r, "r")
    theta = _dev_f64(theta, "theta")
    if theta.numel() != r.numel():
        raise ValueError("r and theta must have the same length")
    nn, mm = (plan.n, plan.m) if plan is not None else (_lib.modes_i32(n), _lib.modes_i32(m))
    J, P = len(nn), r.numel()
    out = torch.empty((max_deriv + 1, J, P), dtype=torch.float64, device=r.device)
    dt = torch.empty((J, P), dtype=torch.float64, device=r.device) if dtheta else None
    st = _stream(r.device)
    with torch.cuda.device(r.device):
        if plan is not None:
            _lib.call("zp_basis_plan", plan.handle, r.data_ptr(), theta.data_ptr(), P, max_deriv, out.data_ptr(),
                      _lib.ptr(dt), st)
        else:
            _lib.call("zp_basis", _lib.i32_ptr(nn), _lib.i32_ptr(mm), J, r.data_ptr(), theta.data_ptr(), P, max_deriv,
                      out.data_ptr(), _lib.ptr(dt), st)
    return out, dt


def radial_per_mode(plan: Plan, r: torch.Tensor) -> torch.Tensor:
    r = _dev_f64(r, "r")
    out = torch.empty((plan.n_modes, r.numel()), dtype=torch.float64, device=r.device)
    with torch.cuda.device(r.device):
        _lib.call("zp_radial_per_mode", plan.handle, r.data_ptr(), r.numel(), out.data_ptr(), _stream(r.device))
    return out


def series_eval(n, m, r, theta, coeffs, prec: str = "fp64emu", plan: Plan | None = None) -> torch.Tensor:
    r = _dev_f64(r, "r")
    theta = _dev_f64(theta, "theta")
    coeffs = _dev_f64(coeffs, "coeffs")
    nn, mm = (plan.n, plan.m) if plan is not None else (_lib.modes_i32(n), _lib.modes_i32(m))
    J, P = len(nn), r.numel()
    if coeffs.dim() != 2 or coeffs.shape[0] != J:
        raise ValueError("coeffs must be [n_modes, n_sets]")
    S = coeffs.shape[1]
    dtype = torch.float64 if prec in ("fp64", "fp64emu") else torch.float32
    out = torch.empty((P, S), dtype=dtype, device=r.device)
    st = _stream(r.device)
    with torch.cuda.device(r.device):
        if plan is not None:
            _lib.call("zp_series_eval_plan", plan.handle, r.data_ptr(), theta.data_ptr(), P, coeffs.data_ptr(), S,
                      PREC[prec], out.data_ptr(), st)
        else:
            _lib.call("zp_series_eval", _lib.i32_ptr(nn), _lib.i32_ptr(mm), J, r.data_ptr(), theta.data_ptr(), P,
                      coeffs.data_ptr(), S, PREC[prec], out.data_ptr(), st)
    return out


def series_adjoint(n, m, r, theta, coeffs, grad_out, need=(True, True, True), plan: Plan | None = None,
                   prec: str = "fp64emu"):
    """(grad_coeffs [J][S], grad_r [P], grad_theta [P]) for upstream grad_out [P][S]; prec
    "fp64emu" (float64-accurate tensor-core contractions, the default) or "fp64" (the DGEMM
    baseline)."""
    if prec not in ("fp64", "fp64emu"):
        raise ValueError("series_adjoint takes prec 'fp64' or 'fp64emu'")
    r = _dev_f64(r, "r")
    theta = _dev_f64(theta, "theta")
    coeffs = _dev_f64(coeffs, "coeffs")
    grad_out = _dev_f64(grad_out, "grad_out")
    nn, mm = (plan.n, plan.m) if plan is not None else (_lib.modes_i32(n), _lib.modes_i32(m))
    J, P = len(nn), r.numel()
    S = coeffs.shape[1]
    if grad_out.shape != (P, S):
        raise ValueError("grad_out must be [n_points, n_sets]")
    dev = r.device
    gC = torch.empty((J, S), dtype=torch.float64, device=dev) if need[0] else None
    gr = torch.empty(P, dtype=torch.float64, device=dev) if need[1] else None
    gt = torch.empty(P, dtype=torch.float64, device=dev) if need[2] else None
    st = _stream(dev)
    with torch.cuda.device(dev):
        if plan is None and prec == "fp64emu":
            _lib.call("zp_series_adjoint", _lib.i32_ptr(nn), _lib.i32_ptr(mm), J, r.data_ptr(), theta.data_ptr(), P,
                      coeffs.data_ptr(), S, grad_out.data_ptr(), _lib.ptr(gC), _lib.ptr(gr), _lib.ptr(gt), st)
        else:
            pl = plan if plan is not None else Plan(nn, mm, device=dev)
            _lib.call("zp_series_adjoint_plan_prec", pl.handle, r.data_ptr(), theta.data_ptr(), P, coeffs.data_ptr(),
                      S, grad_out.data_ptr(), _lib.ptr(gC), _lib.ptr(gr), _lib.ptr(gt), PREC[prec], st)
    return gC, gr, gt


def series_point_hessian(n, m, r, theta, coeffs, grad_out, plan: Plan | None = None):
    """Per-point gradient and 2x2 Hessian block of L = <grad_out, F>: returns
    (grad_r, grad_theta, hess_rr, hess_rt, hess_tt), each [P] float64."""
    r = _dev_f64(r, "r")
    theta = _dev_f64(theta, "theta")
    coeffs = _dev_f64(coeffs, "coeffs")
    G = _dev_f64(grad_out, "grad_out")
    nn, mm = (plan.n, plan.m) if plan is not None else (_lib.modes_i32(n), _lib.modes_i32(m))
    J, P, S = len(nn), r.numel(), coeffs.shape[1]
    if G.shape != (P, S):
        raise ValueError("grad_out must be [n_points, n_sets]")
    outs = [torch.empty(P, dtype=torch.float64, device=r.device) for _ in range(5)]
    ptrs = [o.data_ptr() for o in outs]
    st = _stream(r.device)
    with torch.cuda.device(r.device):
        if plan is not None:
            _lib.call("zp_series_point_hessian_plan", plan.handle, r.data_ptr(), theta.data_ptr(), P, coeffs.data_ptr(),
                      S, G.data_ptr(), *ptrs, st)
        else:
            _lib.call("zp_series_point_hessian", _lib.i32_ptr(nn), _lib.i32_ptr(mm), J, r.data_ptr(), theta.data_ptr(),
                      P, coeffs.data_ptr(), S, G.data_ptr(), *ptrs, st)
    return tuple(outs)


def series_point_hvp(n, m, r, theta, coeffs, grad_out, v_r, v_theta, plan: Plan | None = None):
    """Hessian-vector product of L = <grad_out, F> in the point coordinates for the tangent
    (v_r, v_theta): returns ((Hv)_r, (Hv)_theta), each [P] float64, formed in the library's
    point kernel (the Hessian is block diagonal, one 2x2 block per point)."""
    r = _dev_f64(r, "r")
    theta = _dev_f64(theta, "theta")
    coeffs = _dev_f64(coeffs, "coeffs")
    G = _dev_f64(grad_out, "grad_out")
    v_r = _dev_f64(v_r, "v_r")
    v_theta = _dev_f64(v_theta, "v_theta")
    P, S = r.numel(), coeffs.shape[1]
    if G.shape != (P, S) or v_r.numel() != P or v_theta.numel() != P:
        raise ValueError("grad_out must be [n_points, n_sets] and v_r, v_theta [n_points]")
    pl = plan if plan is not None else Plan(n, m, device=r.device)
    hv_r = torch.empty(P, dtype=torch.float64, device=r.device)
    hv_t = torch.empty(P, dtype=torch.float64, device=r.device)
    with torch.cuda.device(r.device):
        _lib.call("zp_series_point_hvp_plan", pl.handle, r.data_ptr(), theta.data_ptr(), P, coeffs.data_ptr(), S,
                  G.data_ptr(), v_r.data_ptr(), v_theta.data_ptr(), hv_r.data_ptr(), hv_t.data_ptr(),
                  _stream(r.device))
    return hv_r, hv_t


def series_fit(n, m, r, theta, samples, weights=None, ridge: float = 0.0, plan: Plan | None = None,
               prec: str = "fp64emu"):
    """Least-squares coefficients C [J][S] with sum_j Z_j(p) C[j, s] ~ samples[p, s] (weighted,
    optional ridge); float64 results, the Gram matrix and right-hand side by the float64-accurate
    tensor-core GEMM ("fp64emu", the default) or by the DGEMM baseline ("fp64")."""
    if prec not in ("fp64", "fp64emu"):
        raise ValueError("series_fit takes prec 'fp64' or 'fp64emu'")
    r = _dev_f64(r, "r")
    theta = _dev_f64(theta, "theta")
    Y = _dev_f64(samples, "samples")
    w = None if weights is None else _dev_f64(weights, "weights")
    nn, mm = (plan.n, plan.m) if plan is not None else (_lib.modes_i32(n), _lib.modes_i32(m))
    J, P = len(nn), r.numel()
    if Y.dim() != 2 or Y.shape[0] != P:
        raise ValueError("samples must be [n_points, n_sets]")
    S = Y.shape[1]
    out = torch.empty((J, S), dtype=torch.float64, device=r.device)
    st = _stream(r.device)
    with torch.cuda.device(r.device):
        if plan is None and prec == "fp64emu":
            _lib.call("zp_series_fit", _lib.i32_ptr(nn), _lib.i32_ptr(mm), J, r.data_ptr(), theta.data_ptr(),
                      _lib.ptr(w), P, Y.data_ptr(), S, float(ridge), out.data_ptr(), st)
        else:
            pl = plan if plan is not None else Plan(nn, mm, device=r.device)
            _lib.call("zp_series_fit_plan_prec", pl.handle, r.data_ptr(), theta.data_ptr(), _lib.ptr(w), P,
                      Y.data_ptr(), S, float(ridge), out.data_ptr(), PREC[prec], st)
    return out


class ZernikeSeries(torch.autograd.Function):
    """F = Z(r, theta) C with gradients for C, r and theta from the library's adjoint
    (basis recomputed in the backward pass, never stored).  float64 results; prec "fp64emu"
    (float64-accurate tensor-core contractions, the default) or "fp64" (the DGEMM baseline)
    for both passes."""

    @staticmethod
    def forward(ctx, r, theta, coeffs, plan: Plan, prec: str = "fp64emu"):
        if prec not in ("fp64", "fp64emu"):
            raise ValueError("zernike_series takes prec 'fp64' or 'fp64emu'")
        ctx.plan = plan
        ctx.prec = prec
        ctx.save_for_backward(r, theta, coeffs)
        return series_eval(None, None, r, theta, coeffs, prec, plan=plan)

    @staticmethod
    def backward(ctx, grad_out):
        r, theta, coeffs = ctx.saved_tensors
        need = (ctx.needs_input_grad[2], ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        if not any(need):
            return None, None, None, None, None
        gC, gr, gt = series_adjoint(None, None, r, theta, coeffs, grad_out.contiguous(), need=need, plan=ctx.plan,
                                    prec=ctx.prec)
        return gr, gt, gC, None, None


def zernike_series(r, theta, coeffs, plan: Plan, prec: str = "fp64emu") -> torch.Tensor:
    """Differentiable float64 series F[p, s] = sum_j Z_j(r_p, theta_p) coeffs[j, s]."""
    return ZernikeSeries.apply(r, theta, coeffs, plan, prec)


class Batch:
    """Many independent series (uneven mode lists and point counts) evaluated together:
    forward in one persistent launch, adjoint in two (capturable in a CUDA graph).

    instances: list of dicts with keys n, m (host sequences), r, theta (CUDA float64 [P]),
    coeffs (CUDA float64 [J][S]); optional out, grad_out, grad_coeffs, grad_r, grad_theta
    tensors (allocated here when missing).  All instances share n_sets = S."""

    def __init__(self, instances, n_sets: int, out_dtype=torch.float64, with_adjoint: bool = True):
        self._keep = []
        arr = (_lib.ZpInstance * len(instances))()
        self.instances = []
        for i, d in enumerate(instances):
            n = _lib.modes_i32(d["n"])
            m = _lib.modes_i32(d["m"])
            r = _dev_f64(d["r"], "r")
            th = _dev_f64(d["theta"], "theta")
            C = _dev_f64(d["coeffs"], "coeffs")
            P, dev = r.numel(), r.device
            out = d.get("out")
            if out is None:
                out = torch.empty((P, n_sets), dtype=out_dtype, device=dev)
            rec = {"n": n, "m": m, "r": r, "theta": th, "coeffs": C, "out": out}
            if with_adjoint:
                rec["grad_out"] = d.get("grad_out") if d.get("grad_out") is not None else \
                    torch.zeros((P, n_sets), dtype=torch.float64, device=dev)
                for key, shape in (("grad_coeffs", (len(n), n_sets)), ("grad_r", (P,)), ("grad_theta", (P,))):
                    rec[key] = d.get(key) if d.get(key) is not None else \
                        torch.empty(shape, dtype=torch.float64, device=dev)
            self.instances.append(rec)
            a = arr[i]
            a.n, a.m, a.n_modes = _lib.i32_ptr(n), _lib.i32_ptr(m), len(n)
            a.r, a.theta, a.n_points = r.data_ptr(), th.data_ptr(), P
            a.coeffs, a.out = C.data_ptr(), out.data_ptr()
            if with_adjoint:
                a.grad_out = rec["grad_out"].data_ptr()
                a.grad_coeffs = rec["grad_coeffs"].data_ptr()
                a.grad_r = rec["grad_r"].data_ptr()
                a.grad_theta = rec["grad_theta"].data_ptr()
        self.out_dtype = out_dtype
        handle = ctypes.c_void_p()
        _lib.call("zp_batch_create", ctypes.cast(arr, ctypes.c_void_p), len(instances), n_sets, ctypes.byref(handle))
        self.handle = handle
        self._arr = arr

    def forward(self, prec: str = "fp64emu"):
        """F for every instance: "fp64emu" (the fused float64-accurate tensor-core kernel, at most
        16 sets and 5041 modes per instance), "fp64" (float64 contraction on the CUDA cores) or
        "fp32" (float32 contraction, float32 outputs)."""
        code = {"fp64": 0, "fp32": 3, "fp64emu": 4}[prec]
        want = torch.float32 if prec == "fp32" else torch.float64
        if self.out_dtype != want:
            raise TypeError(f"forward({prec!r}) writes {want}, the batch's outputs are {self.out_dtype}")
        _lib.call("zp_batch_forward", self.handle, code, _stream(torch.device("cuda", torch.cuda.current_device())))

    def forward_per_instance(self):
        _lib.call("zp_batch_forward_per_instance", self.handle, 0,
                  _stream(torch.device("cuda", torch.cuda.current_device())))

    def adjoint(self, prec: str = "fp64emu"):
        """grad_coeffs, grad_r, grad_theta for every instance: grad_r and grad_theta by the
        persistent float64 point kernel; grad_coeffs per instance by the float64-accurate
        tensor-core GEMM ("fp64emu") or by the persistent float64 column kernel ("fp64", one
        launch)."""
        code = {"fp64": 0, "fp64emu": 4}[prec]
        _lib.call("zp_batch_adjoint_prec", self.handle, code,
                  _stream(torch.device("cuda", torch.cuda.current_device())))

    def set_config(self, tile_points=128, ctas_per_sm=8, col_ppt=2, col_threads=128):
        _lib.call("zp_batch_set_config", self.handle, tile_points, ctas_per_sm, col_ppt, col_threads)

    def config(self) -> tuple:
        cfg = (ctypes.c_int32 * 4)()
        _lib.call("zp_batch_get_config", self.handle, cfg)
        return tuple(cfg)

    def tune(self, which: str = "forward", prec: str = "fp64", reps: int = 2):
        cfg = (ctypes.c_int32 * 4)()
        best = ctypes.c_float()
        code = {"fp64": 0, "fp32": 3, "fp64emu": 4}[prec]
        _lib.call("zp_batch_tune", self.handle, 0 if which == "forward" else 1, code, reps,
                  _stream(torch.device("cuda", torch.cuda.current_device())), cfg, ctypes.byref(best))
        return tuple(cfg), best.value

    def close(self):
        if getattr(self, "handle", None):
            _lib.call("zp_batch_destroy", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
