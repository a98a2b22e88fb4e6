#!/usr/bin/env python3
"""Benchmark: Zernike basis values per second on the 2601-mode radial workload.

Workload (radial_n100): all (n, m) with 0 <= m <= n <= 100, n - m even (2601 modes), 100000
Chebyshev-Gauss points in [0, 1], radial derivative orders k = 0..3.  One step = one call of
the library's radial walk over the whole batch (plan built once, outside the timed region),
writing 4 x 2601 x 100000 float64 values (8.32 GB).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs the same workload on its own GPU (replicas; the
path has no exchange step) and rank 0 prints the aggregate.  Prints ONE JSON line.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Zernike basis values/s (FP64, points x modes x derivs)"
UNIT = "values/s"
WORKLOAD = "radial_n100"
# Float64 roofline of the walk.  Nominal: 2 float64 lanes per SM per clock (152 SMs x 2 lanes
# x 2 flop x 2.07 GHz = 1.259 TFLOP/s).  The peak the line reports is measured in the run by
# the library's float64 probe (zp_probe_fp64: one wave of independent FMA chains, CUDA events).
SMS, DP_LANES_PER_SM, SM_MAX_MHZ = 152, 2, 2070.0
DP_OPS_PEAK_NOMINAL = SMS * DP_LANES_PER_SM * SM_MAX_MHZ * 1e6
# Algorithmic work per (point, mode) of the k <= 3 radial workload: 14 FMA = 28 flop (the
# unscaled recursion and its three derivative lanes).  The kernel's rescaled form issues 15
# float64 operations per (point, mode): 1 (g) + 1 (g') + 1 + 2 + 3 + 3 (Taylor lanes 0..3) + 4
# (stores scaled by k! w_N), every one as an FMA.
FLOP_PER_VALUE_TUPLE = 28
DP_OPS_PER_VALUE_TUPLE = 15
# DRAM bytes (read + write) of one walk_kernel<3,false,true> launch at 20000 points, from one
# ncu capture of that kernel (dram__bytes_write.sum 1.603925 GB + dram__bytes_read.sum
# 16.961 MB: the output and one read of the power table), scaled to 100000 points (both
# proportional to the point count).  The walk kernel has not changed since that capture (the
# build with the step loop unrolled by eight).
WALK_TRAFFIC_20000 = 1.603924736e9 + 16.96128e6


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-points", type=int, default=1536)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary workloads (series, adjoint, basis latency)")
    ap.add_argument("--series-only", action="store_true",
                    help="run only the mixed_n32 series measurement (profiling captures)")
    ap.add_argument("--series-points", type=int, default=1_000_000)
    ap.add_argument("--series-sets", type=int, default=None,
                    help="with --series-only: fewer coefficient sets (profiling captures of the basis kernel)")
    ap.add_argument("--series-emulated", action="store_true",
                    help="with --series-only: also time the emulated float64 contraction")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the series_n24 forward / adjoint / fit measurement (profiling captures)")
    ap.add_argument("--adjoint-emulated-only", action="store_true",
                    help="run only the series_n24 emulated-float64 adjoint (profiling captures)")
    ap.add_argument("--paper-shapes-only", action="store_true",
                    help="run only the paper-shapes measurement (Algorithm 2, Fig. 3 grid, duplicated modes)")
    ap.add_argument("--fp64-probe-only", action="store_true",
                    help="run only the float64 issue-rate probe (FMA, MUL, ADD) and print its results")
    ap.add_argument("--fused-only", action="store_true",
                    help="run only the fused float64-accurate series measurement (profiling captures)")
    ap.add_argument("--fused-points", type=int, default=1_000_000)
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched forward/adjoint on a reduced batch (profiling captures)")
    ap.add_argument("--batched-adjoint-only", action="store_true",
                    help="run only the batched float64-accurate adjoint (profiling captures)")
    ap.add_argument("--batched-instances", type=int, default=512)
    ap.add_argument("--batched-point-scale", type=float, default=1.0)
    ap.add_argument("--points", type=int, default=100_000,
                    help="point count (smaller values only for profiling captures; the bench line uses 100000)")
    return ap.parse_args()


def workload(n_points: int = 100_000):
    from paper_2409_19156_gb300 import inputs

    ns, ms = inputs.radial_modes(100)
    r = inputs.chebyshev_gauss_points(n_points)
    return ns, ms, r


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.tmp,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.tmp.read())) if len(r) >= 9]
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: power above the midpoint between idle and peak draw
        thr = min(power) + 0.5 * (max(power) - min(power))
        loaded = [s for s, p in zip(sm, power) if p >= thr] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ----------------------------------------------------------------------------- oracle timing
def _oracle_chunk(args):
    ns, ms, rs = args
    from oracle import radial as oradial

    tab = oradial.radial_table(ns, ms, rs, 3)
    return len(ns) * len(rs) * 4 + 0 * len(tab)


def _oracle_parity_chunk(args):
    """Exact oracle values at a few points against the GPU's values there: per derivative
    order k, the largest absolute error and the largest error over the tolerance
    1e-11 max(n, 1)^(2k)."""
    ns, ms, rs, gpu = args
    import numpy as np

    from oracle import radial as oradial

    want = np.array(oradial.radial_table(ns, ms, rs, 3))  # [4][modes][points]
    err = np.abs(np.asarray(gpu) - want)
    n1 = np.maximum(np.asarray(ns, dtype=np.float64), 1.0)
    tol = np.stack([1e-11 * n1 ** (2 * k) for k in range(4)])[:, :, None]
    return err.max(axis=(1, 2)).tolist(), float((err / tol).max())


class OraclePool:
    """A spawn-started process pool over the host cores that times the exact CPU oracle on a
    sample of the workload's points (all modes, k = 0..3)."""

    def __init__(self, cores: int | None = None):
        import multiprocessing as mp

        self.cores = cores or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores)
        ns, ms, self.r = workload()
        self.ns, self.ms = [int(v) for v in ns], [int(v) for v in ms]
        self.pool.map(_oracle_chunk, [(self.ns[:3], self.ms[:3], [0.5])] * self.cores)  # start-up

    def time(self, n_points: int) -> dict:
        import numpy as np

        idx = ((len(self.r) - 1) * (0.5 + 0.5 * np.cos(np.pi * (np.arange(n_points) + 0.5) / n_points))).astype(int)
        pts = [float(self.r[i]) for i in idx]
        chunks = [c for c in (pts[i::self.cores] for i in range(self.cores)) if c]
        t0 = time.perf_counter()
        vals = sum(self.pool.map(_oracle_chunk, [(self.ns, self.ms, c) for c in chunks]))
        dt = time.perf_counter() - t0
        return {"value": vals / dt, "unit": UNIT, "cores": len(chunks), "kind": "oracle",
                "sample": f"{len(pts)} of the 100000 points x all 2601 modes x k=0..3 "
                          f"({vals} exact-rational values in {dt:.2f} s)"}

    def parity(self, rs, gpu) -> dict:
        """The GPU output of the timed workload (gpu: [4][modes][len(rs)] at the points rs)
        against the exact oracle, the points dealt over the pool."""
        import numpy as np

        gpu = np.asarray(gpu)
        parts = [list(range(i, len(rs), self.cores)) for i in range(self.cores)]
        parts = [q for q in parts if q]
        res = self.pool.map(_oracle_parity_chunk, [(self.ns, self.ms, [float(rs[i]) for i in q], gpu[:, :, q])
                                                   for q in parts])
        max_abs = [max(r[0][k] for r in res) for k in range(4)]
        worst = max(r[1] for r in res)
        return {"points": len(rs), "values": int(gpu.size), "max_abs_err_k0_k3": max_abs,
                "max_err_over_tol": worst, "tol": "1e-11 * max(n,1)^(2k)", "ok": worst <= 1.0}

    def time_alg1_numpy(self, chunk: int = 8192) -> dict:
        """The numpy restatement of Algorithm 1 on the whole workload (all 100000 points, all
        2601 modes, k = 0..3), the m-columns dealt round-robin over the pool's processes, each
        process writing its columns' values chunk by chunk (not a timing of the oracle)."""
        import numpy as np

        r = np.asarray(self.r, dtype=np.float64)
        cols = sorted(set(abs(m) for m in self.ms))
        parts = [cols[i::self.cores] for i in range(self.cores)]
        parts = [p for p in parts if p]
        t0 = time.perf_counter()
        vals = sum(self.pool.map(_alg1_numpy_chunk, [(r, 100, p, chunk) for p in parts]))
        dt = time.perf_counter() - t0
        return {"value": vals / dt, "unit": UNIT, "cores": len(parts), "kind": "numpy Algorithm 1",
                "sample": f"whole workload: {vals} values in {dt:.2f} s, {chunk}-point chunks"}

    def close(self):
        self.pool.close()
        self.pool.join()


def alg1_numpy_column(r, n_max: int, m: int):
    """Algorithm 1 restated in numpy for one m-column, the CPU comparison program: R_n^m and
    its first three rho-derivatives for n = m, m+2, ..., n_max at the points r, returned as a
    [4][(n_max-m)//2 + 1][len(r)] float64 block.  Seeds rho^m and ((m+2) rho^2 - (m+1)) rho^m
    (Sec. 3, the first two Jacobi polynomials times (-1)^N rho^m), then the Jacobi three-term
    recursion of Sec. 3 in rho^2 form, R_N = (2 a_N rho^2 - a_N - b_N) R_{N-1} - c_N R_{N-2},
    differentiated term by term in rho (Leibniz on the factor g = 2 a_N rho^2 - a_N - b_N)."""
    import numpy as np

    r = np.asarray(r, dtype=np.float64)
    n_steps = (n_max - m) // 2
    out = np.empty((4, n_steps + 1, r.size))

    def falling(p, k):
        v = 1
        for i in range(k):
            v *= p - i
        return v

    def power_deriv(p, k):  # d^k/drho^k rho^p
        return falling(p, k) * r ** (p - k) if k <= p else np.zeros_like(r)

    for k in range(4):
        out[k, 0] = power_deriv(m, k)
        if n_steps >= 1:
            out[k, 1] = (m + 2) * power_deriv(m + 2, k) - (m + 1) * power_deriv(m, k)
    u = r * r
    for N in range(2, n_steps + 1):
        D = 2.0 * N * (N + m) * (2 * N + m - 2)
        a = (2 * N + m - 1) * (2 * N + m) * (2 * N + m - 2) / D
        b = (2 * N + m - 1) * m * m / D
        c = 2.0 * (N + m - 1) * (N - 1) * (2 * N + m) / D
        g = 2.0 * a * u - (a + b)
        g1 = 4.0 * a * r
        g2 = 4.0 * a
        p0, p1, p2, p3 = out[0, N - 1], out[1, N - 1], out[2, N - 1], out[3, N - 1]
        out[0, N] = g * p0 - c * out[0, N - 2]
        out[1, N] = g * p1 + g1 * p0 - c * out[1, N - 2]
        out[2, N] = g * p2 + 2.0 * g1 * p1 + g2 * p0 - c * out[2, N - 2]
        out[3, N] = g * p3 + 3.0 * g1 * p2 + 3.0 * g2 * p1 - c * out[3, N - 2]
    return out


def _alg1_numpy_chunk(args):
    r, n_max, m_list, chunk = args
    values = 0
    for lo in range(0, len(r), chunk):
        rr = r[lo:lo + chunk]
        for m in m_list:
            values += alg1_numpy_column(rr, n_max, m).size
    return values


def time_oracle(n_points: int, cores: int | None = None) -> dict:
    pool = OraclePool(cores)
    try:
        return pool.time(n_points)
    finally:
        pool.close()


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest of every rank's x (x itself when not distributed)."""
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(units_per_rank_step: float, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank's units in one step over the slowest rank's step time."""
    return world * units_per_rank_step / (ms_per_step * 1e-3)


# ----------------------------------------------------------------------------- our arm
def run_ours(args) -> None:
    import numpy as np
    import torch

    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ns, ms, r = workload(args.points)
    J, P, K = len(ns), len(r), 4
    dev = torch.device("cuda", local)
    plan = zp.Plan(ns, ms, device=dev)
    rt = torch.as_tensor(r, device=dev)
    out = torch.empty((K, J, P), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 2x L2
    lib = _lib.load()
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step():
        st = lib.zp_radial_plan(plan.handle, rt.data_ptr(), P, 3, out.data_ptr(), sp)
        if st:
            _lib.check("zp_radial_plan", st)

    for _ in range(args.warmup):
        step()
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ms_steps = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # Sampled output of the timed steps (every point index spread over [0, 1] and both ends),
    # checked against the exact oracle in the CPU-baseline leg below.
    parity_idx = np.unique(np.concatenate([[0, P - 1], np.linspace(0, P - 1, 62).astype(int)]))
    parity_gpu = out[:, :, torch.as_tensor(parity_idx, device=dev)].cpu().numpy()
    total_ms = max_over_ranks(sum(ms_steps), dist, dev)
    ms_per_step = total_ms / args.steps
    values_per_step = P * J * K
    value = aggregate_value(values_per_step, world, ms_per_step)

    # Roofline of the walk kernel (float64-issue bound), the dominant of the step's two
    # launches (point preparation, walk): its own device time from the timed entry point,
    # which records CUDA events around each launch on this stream.
    import ctypes

    phase = (ctypes.c_float * 2)()
    prep_ms, walk_ms = [], []
    for i in range(10):
        flush.fill_(i & 0xFF)
        _lib.check("zp_radial_plan_timed", lib.zp_radial_plan_timed(plan.handle, rt.data_ptr(), P, 3, out.data_ptr(),
                                                                     sp, phase))
        prep_ms.append(phase[0])
        walk_ms.append(phase[1])
    dp_ops = DP_OPS_PER_VALUE_TUPLE * P * J
    flops = FLOP_PER_VALUE_TUPLE * P * J
    kernel_ms = statistics.mean(walk_ms)
    achieved = dp_ops / (kernel_ms * 1e-3)
    achieved_flops = flops / (kernel_ms * 1e-3)
    out_bytes = values_per_step * 8
    # The float64 peak, measured now on this GPU: best of three probe launches per operation.
    probe = {}
    for op, name in ((0, "fma"), (1, "mul"), (2, "add")):
        best = None
        for _ in range(3):
            res = (ctypes.c_double * 6)()
            _lib.check("zp_probe_fp64", lib.zp_probe_fp64(op, 20000, sp, res))
            if best is None or res[2] > best[2]:
                best = list(res)
        probe[name] = {"ops_per_s": best[2], "lanes_per_sm_clk": best[3], "implied_sm_mhz": best[4], "ms": best[1]}
    fma_ops = probe["fma"]["ops_per_s"]
    peak_flops = 2.0 * fma_ops
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    # End to end through the C ABI with host buffers: r from pinned host memory in, the
    # whole result back to pinned host memory, every step.
    e2e = None
    if args.e2e_steps > 0:
        r_host = torch.as_tensor(r).pin_memory()
        out_host = torch.empty((K, J, P), dtype=torch.float64, pin_memory=True)
        rt2 = torch.empty_like(rt)

        def e2e_copy_step():
            # inputs H2D, kernel into device memory, whole result D2H
            rt2.copy_(r_host, non_blocking=True)
            st = lib.zp_radial_plan(plan.handle, rt2.data_ptr(), P, 3, out.data_ptr(), sp)
            if st:
                _lib.check("zp_radial_plan", st)
            out_host.copy_(out, non_blocking=True)

        def e2e_mapped_step():
            # inputs H2D, kernel writing the result straight into pinned (mapped) host memory
            rt2.copy_(r_host, non_blocking=True)
            st = lib.zp_radial_plan(plan.handle, rt2.data_ptr(), P, 3, out_host.data_ptr(), sp)
            if st:
                _lib.check("zp_radial_plan", st)

        def e2e_host_buffers_step():
            # one C-ABI call on host buffers: the kernels read r from pinned host memory and write
            # the result into pinned host memory, both across the host link
            st = lib.zp_radial_plan(plan.handle, r_host.data_ptr(), P, 3, out_host.data_ptr(), sp)
            if st:
                _lib.check("zp_radial_plan", st)

        def time_e2e(fn):
            fn()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.e2e_steps):
                fn()
            e1.record(stream)
            barrier()
            return max_over_ranks(e0.elapsed_time(e1) / args.e2e_steps, dist, dev)

        streams = [torch.cuda.Stream(dev) for _ in range(4)]
        flat_dev, flat_host = out.view(-1), out_host.view(-1)
        chunk = (flat_dev.numel() + 3) // 4

        def e2e_multi_copy_step():
            # inputs H2D, kernel into device memory, result D2H split over four copy streams
            rt2.copy_(r_host, non_blocking=True)
            st = lib.zp_radial_plan(plan.handle, rt2.data_ptr(), P, 3, out.data_ptr(), sp)
            if st:
                _lib.check("zp_radial_plan", st)
            done = torch.cuda.Event()
            done.record(stream)
            for i, cs in enumerate(streams):
                cs.wait_event(done)
                with torch.cuda.stream(cs):
                    flat_host[i * chunk:(i + 1) * chunk].copy_(flat_dev[i * chunk:(i + 1) * chunk], non_blocking=True)
            for cs in streams:
                stream.wait_stream(cs)

        t_copy = time_e2e(e2e_copy_step)
        t_multi = time_e2e(e2e_multi_copy_step)
        assert float(out_host[3, J - 1, P - 1]) == float(out[3, J - 1, P - 1].item())
        assert float(out_host[3, J - 1, P - 1]) == float(out[3, J - 1, P - 1].item())
        t_mapped = time_e2e(e2e_mapped_step)
        assert float(out_host[3, J - 1, P - 1]) == float(out[3, J - 1, P - 1].item())
        out_host.zero_()
        t_host = time_e2e(e2e_host_buffers_step)
        assert float(out_host[3, J - 1, P - 1]) == float(out[3, J - 1, P - 1].item())
        # The end-to-end figure is the C-ABI call on host buffers; the other forms are context.
        best, how = t_host, "one C-ABI call on pinned host buffers (r read and result written across the link)"
        e2e = {"value": aggregate_value(values_per_step, world, best), "unit": UNIT,
               "h2d_bytes_per_step": P * 8, "d2h_bytes_per_step": out_bytes, "ms_per_step": best, "how": how,
               "ms_per_step_copy": t_copy, "ms_per_step_copy4": t_multi, "ms_per_step_mapped": t_mapped,
               "ms_per_step_host_buffers": t_host}

    extras = None
    # The secondary workloads run only in a single-GPU job: under torchrun every rank runs the
    # headline workload alone.
    if world == 1 and not args.no_extras:
        del out
        torch.cuda.empty_cache()
        extras = {"series": measure_series(dev, peaks), "adjoint": measure_adjoint(dev),
                  "basis": measure_basis_latency(dev), "batched": measure_batched(dev),
                  "fused_series": measure_fused_series(dev, peaks),
                  "paper_shapes": measure_paper_shapes(dev)}

    cpu = cpu_alg1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool()
        try:
            cpu = pool.time(args.cpu_sample_points)
            cpu["parity_of_the_timed_output"] = pool.parity(np.asarray(r)[parity_idx], parity_gpu)
            cpu_alg1 = pool.time_alg1_numpy()
        finally:
            pool.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "modes": J, "n_max": 100, "points": P, "derivs": K,
                       "points_dist": "Chebyshev-Gauss nodes mapped to [0,1]", "parallelism": f"replicas{world}",
                       "l2": "256 MB write between steps, outside the per-step CUDA events; each step writes 8.3 GB"},
            "roofline": {"bound": "alu", "achieved": achieved_flops / 1e12, "peak": peak_flops / 1e12,
                         "unit": "TFLOP/s", "frac": achieved_flops / peak_flops,
                         "traffic": WALK_TRAFFIC_20000 * P / 20000 if WALK_TRAFFIC_20000 else None,
                         "traffic_note": "ncu dram__bytes_read+write of a 20000-point launch scaled by points",
                         "kernel": "walk_kernel<3,false,true>", "flop_per_launch": flops,
                         "flop_per_unit": FLOP_PER_VALUE_TUPLE, "units_per_launch": P * J,
                         "kernel_ms": kernel_ms, "point_prep_kernel_ms": statistics.mean(prep_ms),
                         "peak_source": "measured in this run: zp_probe_fp64 float64 FMA rate x 2 flop "
                                        "(best of 3 one-wave launches, CUDA events)",
                         "fp64_probe": probe,
                         "peak_nominal": DP_OPS_PEAK_NOMINAL * 2 / 1e12,
                         "frac_of_nominal": achieved_flops / (2 * DP_OPS_PEAK_NOMINAL),
                         "issued_ops_per_unit": DP_OPS_PER_VALUE_TUPLE,
                         "issued_ops_frac_of_measured_fma_rate": achieved / fma_ops,
                         "hbm_write_gbs": out_bytes / (kernel_ms * 1e-3) / 1e9,
                         "hbm_frac_of_measured_copy": out_bytes / (kernel_ms * 1e-3) / 1e9 / hbm_peak},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "cpu_alg1_numpy": cpu_alg1,
            "clocks": clk,
            "gpu_launches": 2 * args.steps,  # point_prep_kernel + walk_kernel per step
            "wall_s_timed": wall,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- secondary workloads
def _events_ms(stream, fn, steps):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def measure_series(dev, peaks, steps: int = 3, n_points: int = 1_000_000, with_fp64: bool = True,
                   with_emulated_only: bool = False, n_sets: int | None = None) -> dict:
    """mixed_n32: 561 modes, 1e6 points r = sqrt(U), 4096 coefficient sets.  The split-precision
    tensor-core series (per-phase CUDA-event times recorded by the library on the launching
    stream) against the plain float64 basis-then-DGEMM form on the same inputs."""
    import ctypes

    import torch

    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import _lib, inputs

    cfg = inputs.WORKLOADS["mixed_n32"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.sqrt_uniform_points(cfg["n_points"], cfg["seed"])
    r, th = r[:n_points], th[:n_points]
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    if n_sets is not None:
        C = C[:, :n_sets].copy()
    J, P, S = len(ns), len(r), C.shape[1]
    plan = zp.Plan(ns, ms, device=dev)
    rt, tt, Ct = (torch.as_tensor(x, device=dev) for x in (r, th, C))
    lib = _lib.load()
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    out = {"workload": "mixed_n32", "modes": J, "points": P, "sets": S}
    F = torch.empty((P, S), dtype=torch.float32, device=dev)
    phase = (ctypes.c_float * 3)()
    bf16_peak = peaks.get("bf16_tflops", 1906.3) * 1e12
    for prec, code, parts, bk in (("bf16x3", 1, 3, 64), ("tf32", 2, 1, 32)):
        kp = -(-J // bk) * bk
        issued = parts * 2.0 * (-(-P // 128) * 128) * kp * (-(-S // 256) * 256)
        runs = []
        for i in range(steps + 1):
            t = _events_ms(stream, lambda: _lib.check("zp_series_eval_timed", lib.zp_series_eval_timed(
                plan.handle, rt.data_ptr(), tt.data_ptr(), P, Ct.data_ptr(), S, code, F.data_ptr(), sp, phase)), 1)
            if i:
                runs.append((t, list(phase)))
        ph = [statistics.mean(x[1][k] for x in runs) for k in range(3)]
        # Whole-call time through the untimed entry point (the timed one synchronises).
        call_ms = _events_ms(stream, lambda: _lib.check("zp_series_eval_plan", lib.zp_series_eval_plan(
            plan.handle, rt.data_ptr(), tt.data_ptr(), P, Ct.data_ptr(), S, code, F.data_ptr(), sp)), steps)
        _lib.check("zp_device_wait_status", lib.zp_device_wait_status(1))
        peak = bf16_peak if prec == "bf16x3" else bf16_peak / 2  # TF32 dense rate = bf16 / 2 (nominal ratio)
        out[prec] = {"ms_per_call": call_ms, "ms_coeff_split": ph[0], "ms_basis_split": ph[1], "ms_gemm": ph[2],
                     "useful_tflops": 2.0 * P * J * S / (call_ms * 1e-3) / 1e12,
                     "roofline": {"bound": "tensor", "kernel": f"split_gemm_kernel<{prec}>",
                                  "achieved": issued / (ph[2] * 1e-3) / 1e12, "peak": peak / 1e12,
                                  "unit": "TFLOP/s", "frac": issued / (ph[2] * 1e-3) / peak,
                                  "flops_per_call_issued": issued,
                                  "peak_source": "MEASURED_PEAKS bf16_tflops (burst)" +
                                                 (" x 1/2 (nominal tf32:bf16)" if prec == "tf32" else "")}}
        if prec == "bf16x3":
            F_keep = F.clone()
    if with_emulated_only:
        Fe = torch.empty((P, S), dtype=torch.float64, device=dev)
        emu = lambda: _lib.check("zp_series_eval_plan", lib.zp_series_eval_plan(  # noqa: E731
            plan.handle, rt.data_ptr(), tt.data_ptr(), P, Ct.data_ptr(), S, 4, Fe.data_ptr(), sp))
        emu()
        out["fp64_emulated_ms"] = _events_ms(stream, emu, steps)
        del Fe
    if not with_fp64:
        return out
    # Plain float64 form: basis to HBM, then cuBLAS DGEMM.
    zp.series_eval(None, None, rt[:1024].contiguous(), tt[:1024].contiguous(), Ct, "fp64", plan=plan)
    torch.cuda.synchronize()
    F64 = torch.empty((P, S), dtype=torch.float64, device=dev)
    t64 = _events_ms(stream, lambda: _lib.check("zp_series_eval_plan", lib.zp_series_eval_plan(
        plan.handle, rt.data_ptr(), tt.data_ptr(), P, Ct.data_ptr(), S, 0, F64.data_ptr(), sp)), 1)
    num = den = 0.0
    for i in range(0, P, 1 << 17):
        d = F_keep[i:i + (1 << 17)].double() - F64[i:i + (1 << 17)]
        num += float((d * d).sum())
        den += float((F64[i:i + (1 << 17)] ** 2).sum())
    # float64-accurate contraction emulated on the tensor cores (error-free slicing)
    del F_keep
    Fe = torch.empty((P, S), dtype=torch.float64, device=dev)
    emu = lambda: _lib.check("zp_series_eval_plan", lib.zp_series_eval_plan(  # noqa: E731
        plan.handle, rt.data_ptr(), tt.data_ptr(), P, Ct.data_ptr(), S, 4, Fe.data_ptr(), sp))
    emu()
    t_emu = _events_ms(stream, emu, 1)
    out["fp64_emulated_ms"] = t_emu
    out["fp64_emulated_max_abs_diff_vs_dgemm"] = max(float((Fe[i:i + (1 << 17)] - F64[i:i + (1 << 17)]).abs().max())
                                                     for i in range(0, P, 1 << 17))
    out["speedup_fp64_emulated_vs_dgemm"] = t64 / t_emu
    del Fe
    F_keep = None
    out["fp64_basis_then_dgemm_ms"] = t64
    out["speedup_bf16x3_vs_fp64"] = t64 / out["bf16x3"]["ms_per_call"]
    out["bf16x3_rel_frobenius_vs_fp64"] = math.sqrt(num / den)
    del F64, F
    torch.cuda.empty_cache()
    return out


def measure_adjoint(dev, steps: int = 5) -> dict:
    """series_n24: 325 modes, 250 x 200 polar grid, 256 sets; float64 forward and adjoint."""
    import torch

    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import inputs

    cfg = inputs.WORKLOADS["series_n24"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.polar_grid(cfg["n_r"], cfg["n_theta"])
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    G = torch.randn((len(r), C.shape[1]), dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(2))
    plan = zp.Plan(ns, ms, device=dev)
    rt, tt, Ct = (torch.as_tensor(x, device=dev) for x in (r, th, C))
    stream = torch.cuda.current_stream(dev)
    # "fp64": the plain basis-then-DGEMM baseline; "fp64emu": the library's default float64 path.
    zp.series_eval(None, None, rt, tt, Ct, "fp64", plan=plan)
    zp.series_adjoint(None, None, rt, tt, Ct, G, plan=plan, prec="fp64")
    fwd = _events_ms(stream, lambda: zp.series_eval(None, None, rt, tt, Ct, "fp64", plan=plan), steps)
    zp.series_eval(None, None, rt, tt, Ct, "fp64emu", plan=plan)
    fwd_emu = _events_ms(stream, lambda: zp.series_eval(None, None, rt, tt, Ct, "fp64emu", plan=plan), steps)
    adj = _events_ms(stream, lambda: zp.series_adjoint(None, None, rt, tt, Ct, G, plan=plan, prec="fp64"), steps)
    zp.series_adjoint(None, None, rt, tt, Ct, G, plan=plan, prec="fp64emu")
    adj_emu = _events_ms(stream, lambda: zp.series_adjoint(None, None, rt, tt, Ct, G, plan=plan, prec="fp64emu"),
                         steps)
    # Least-squares fit of the same coefficients back from the series values, with the
    # grid's exact quadrature weights (Gauss-Legendre in r^2 x uniform theta).
    import numpy as np

    _, wgl = np.polynomial.legendre.leggauss(cfg["n_r"])
    w = torch.as_tensor(np.repeat(0.25 * wgl, cfg["n_theta"]) * (2.0 * math.pi / cfg["n_theta"]), device=dev)
    Y = zp.series_eval(None, None, rt, tt, Ct, plan=plan)
    Cfit = zp.series_fit(None, None, rt, tt, Y, weights=w, plan=plan, prec="fp64")
    t0 = time.perf_counter()
    for _ in range(steps):
        zp.series_fit(None, None, rt, tt, Y, weights=w, plan=plan, prec="fp64")
    fit_ms = (time.perf_counter() - t0) * 1e3 / steps  # the fit synchronises its stream
    Cfit_emu = zp.series_fit(None, None, rt, tt, Y, weights=w, plan=plan, prec="fp64emu")
    t0 = time.perf_counter()
    for _ in range(steps):
        zp.series_fit(None, None, rt, tt, Y, weights=w, plan=plan, prec="fp64emu")
    fit_emu_ms = (time.perf_counter() - t0) * 1e3 / steps
    return {"workload": "series_n24", "modes": len(ns), "points": len(r), "sets": C.shape[1],
            "baseline": "fp64_* = float64 basis then cuBLAS DGEMM; fp64_emulated_* = the default path",
            "fp64_forward_ms": fwd, "fp64_emulated_forward_ms": fwd_emu, "fp64_adjoint_ms": adj,
            "fp64_emulated_adjoint_ms": adj_emu, "fp64_fit_ms": fit_ms, "fp64_emulated_fit_ms": fit_emu_ms,
            "fit_roundtrip_max_abs_err": float((Cfit - Ct).abs().max()),
            "fit_emulated_roundtrip_max_abs_err": float((Cfit_emu - Ct).abs().max())}


def measure_adjoint_emulated(dev, steps: int = 2) -> dict:
    """series_n24 emulated-float64 adjoint alone (one warm-up call, then `steps` timed calls)."""
    import torch

    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import inputs

    cfg = inputs.WORKLOADS["series_n24"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.polar_grid(cfg["n_r"], cfg["n_theta"])
    C = inputs.scaled_normal_coeffs(ns, cfg["n_sets"], cfg["seed"])
    G = torch.randn((len(r), C.shape[1]), dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(2))
    plan = zp.Plan(ns, ms, device=dev)
    rt, tt, Ct = (torch.as_tensor(x, device=dev) for x in (r, th, C))
    stream = torch.cuda.current_stream(dev)
    zp.series_adjoint(None, None, rt, tt, Ct, G, plan=plan, prec="fp64emu")
    ms_ = _events_ms(stream, lambda: zp.series_adjoint(None, None, rt, tt, Ct, G, plan=plan, prec="fp64emu"), steps)
    return {"workload": "series_n24", "fp64_emulated_adjoint_ms": ms_}


def fused_fp64_ops(ns, ms) -> int:
    """float64 operations per point of the fused kernel's walk: per column step N >= 2 the
    recursion (2), per step with outputs the weight product (1), per output the angular product
    (1); per column the angle addition (4)."""
    cols = {}
    for n, m in zip(ns, ms):
        cols.setdefault(abs(int(m)), {}).setdefault((int(n) - abs(int(m))) // 2, 0)
        cols[abs(int(m))][(int(n) - abs(int(m))) // 2] += 1
    ops = 0
    for m, steps in cols.items():
        n_steps = max(steps) + 1
        ops += 4 + 2 * max(0, n_steps - 2)
        ops += sum(1 + c for c in steps.values())
    return ops


def measure_fused_series(dev, peaks, steps: int = 5, n_points: int = 1_000_000) -> dict:
    """The fused float64-accurate series (basis on chip, 16 sets) on the mixed_n32 points (561
    modes, 1e6 points r = sqrt(U)) against the plain float64 basis-then-DGEMM form, with the
    fused kernel's float64 roofline (its walk issues fused_fp64_ops per point)."""
    import ctypes

    import numpy as np
    import torch

    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import _lib, inputs

    cfg = inputs.WORKLOADS["mixed_n32"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.sqrt_uniform_points(n_points, cfg["seed"])
    S = 16
    C = inputs.scaled_normal_coeffs(ns, S, cfg["seed"])
    plan = zp.Plan(ns, ms, device=dev)
    rt, tt, Ct = (torch.as_tensor(x, device=dev) for x in (r, th, C))
    stream = torch.cuda.current_stream(dev)
    lib = _lib.load()
    out = torch.empty((n_points, S), dtype=torch.float64, device=dev)
    out64 = torch.empty_like(out)
    sp = stream.cuda_stream

    def run(code, o):
        _lib.check("zp_series_eval_plan", lib.zp_series_eval_plan(plan.handle, rt.data_ptr(), tt.data_ptr(), n_points,
                                                                   Ct.data_ptr(), S, code, o.data_ptr(), sp))

    run(4, out)
    t_fused = _events_ms(stream, lambda: run(4, out), steps)
    run(0, out64)
    t_dgemm = _events_ms(stream, lambda: run(0, out64), 2)
    ops = fused_fp64_ops(ns, ms) * n_points
    probe = (ctypes.c_double * 6)()
    _lib.check("zp_probe_fp64", lib.zp_probe_fp64(0, 20000, sp, probe))
    diff = float((out - out64).abs().max())
    # The adjoint of the same series (grad_C, grad_r, grad_theta): the default path (grad_C by the
    # emulated GEMM, the point gradients from the fused derivative series) against the float64
    # basis + DGEMM form (H = C G^T through HBM).
    G = torch.as_tensor(np.random.default_rng(cfg["seed"]).standard_normal((n_points, S)), device=dev)
    gC = torch.empty((len(ns), S), dtype=torch.float64, device=dev)
    gr = torch.empty(n_points, dtype=torch.float64, device=dev)
    gt = torch.empty_like(gr)
    res = [(gC.clone(), gr.clone(), gt.clone()) for _ in range(2)]

    def adj(code, o):
        _lib.check("zp_series_adjoint_plan_prec", lib.zp_series_adjoint_plan_prec(
            plan.handle, rt.data_ptr(), tt.data_ptr(), n_points, Ct.data_ptr(), S, G.data_ptr(), o[0].data_ptr(),
            o[1].data_ptr(), o[2].data_ptr(), code, sp))

    adj(4, res[0])
    t_adj_emu = _events_ms(stream, lambda: adj(4, res[0]), 3)
    adj(0, res[1])
    t_adj_64 = _events_ms(stream, lambda: adj(0, res[1]), 2)
    adj_diff = [float((a - b).abs().max() / (1.0 + b.abs().max())) for a, b in zip(res[0], res[1])]
    del G, res
    return {"workload": "mixed_n32 points, 16 sets", "modes": len(ns), "points": n_points, "sets": S,
            "fp64emu_fused_ms": t_fused, "fp64_basis_then_dgemm_ms": t_dgemm,
            "speedup_fused_vs_basis_then_dgemm": t_dgemm / t_fused,
            "fp64emu_adjoint_ms": t_adj_emu, "fp64_dgemm_adjoint_ms": t_adj_64,
            "speedup_emulated_vs_dgemm_adjoint": t_adj_64 / t_adj_emu,
            "adjoint_rel_diff_vs_dgemm_gC_gr_gt": adj_diff,
            "max_abs_diff_vs_dgemm": diff, "max_abs_value": float(out64.abs().max()),
            "roofline": {"bound": "alu", "kernel": "fused_emu_kernel (includes the coefficient digit kernels)",
                         "fp64_ops": ops, "achieved_ops_per_s": ops / (t_fused * 1e-3),
                         "peak_ops_per_s": probe[2], "frac": ops / (t_fused * 1e-3) / probe[2],
                         "peak_source": "zp_probe_fp64 float64 FMA rate measured in this run"}}


def measure_paper_shapes(dev, steps: int = 50) -> dict:
    """The paper's own timing shapes.  (1) Algorithm 2 (one recursion per mode) against the
    per-column walk (Algorithm 1's decomposition) on the 2601-mode radial set, k = 0, 100000
    points.  (2) The Fig. 3 grid: full radial set k = 0 at 100 and 1000 linearly spaced points
    for n_max = 10, 20, 50, 100, as single calls and as CUDA-graph replays.  (3) Duplicated
    modes, 16 copies of each mode of the n <= 24 set."""
    import numpy as np
    import torch

    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import _lib, inputs

    lib = _lib.load()
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    ns, ms = inputs.radial_modes(100)
    r = torch.as_tensor(inputs.chebyshev_gauss_points(100_000), device=dev)
    plan = zp.Plan(ns, ms, device=dev)
    out = torch.empty((len(ns), r.numel()), dtype=torch.float64, device=dev)
    walk = lambda: _lib.check("zp_radial_plan", lib.zp_radial_plan(plan.handle, r.data_ptr(), r.numel(), 0,  # noqa: E731
                                                                     out.data_ptr(), sp))
    per_mode = lambda: _lib.check("zp_radial_per_mode", lib.zp_radial_per_mode(  # noqa: E731
        plan.handle, r.data_ptr(), r.numel(), out.data_ptr(), sp))
    walk()
    per_mode()
    res = {"alg1_column_walk_k0_ms": _events_ms(stream, walk, 5), "alg2_per_mode_k0_ms": _events_ms(stream, per_mode, 2)}
    res["alg2_over_alg1"] = res["alg2_per_mode_k0_ms"] / res["alg1_column_walk_k0_ms"]
    del out
    fig3 = []
    for P in (100, 1000):
        rr = torch.as_tensor(inputs.linspace_points(P), device=dev)
        for n_max in (10, 20, 50, 100):
            n2, m2 = inputs.radial_modes(n_max)
            pl = zp.Plan(n2, m2, device=dev)
            o = torch.empty((len(n2), P), dtype=torch.float64, device=dev)
            call = lambda: _lib.check("zp_radial_plan", lib.zp_radial_plan(  # noqa: E731
                pl.handle, rr.data_ptr(), P, 0, o.data_ptr(), torch.cuda.current_stream(dev).cuda_stream))
            call()
            t_call = _events_ms(stream, call, steps)
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream(dev)
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                with torch.cuda.graph(g, stream=side):
                    call()
            stream.wait_stream(side)
            g.replay()
            t_graph = _events_ms(stream, g.replay, steps)
            fig3.append({"points": P, "n_max": n_max, "modes": len(n2), "us_per_call": t_call * 1e3,
                         "us_per_graph_replay": t_graph * 1e3})
    res["fig3_full_radial_set_k0"] = fig3
    # Duplicated modes (the Zernike x Fourier footnote of Sec. 3): the full n <= 24 set, every
    # mode repeated L = 16 times, Z at k = 0 on 100000 points.  One recursion per distinct
    # column, 16 stores per value: the launch is bound by the HBM writes.
    n24, m24 = inputs.full_zernike_modes(24)
    L = 16
    nd, md = np.repeat(n24, L), np.repeat(m24, L)
    rd, td = (torch.as_tensor(a, device=dev) for a in inputs.uniform_points(100_000, 17))
    pld = zp.Plan(nd, md, device=dev)
    od = torch.empty((len(nd), rd.numel()), dtype=torch.float64, device=dev)
    dup = lambda: _lib.check("zp_basis_plan", lib.zp_basis_plan(  # noqa: E731
        pld.handle, rd.data_ptr(), td.data_ptr(), rd.numel(), 0, od.data_ptr(), None, sp))
    dup()
    t_dup = _events_ms(stream, dup, 5)
    wbytes = od.numel() * 8
    res["duplicated_modes_n24_x16"] = {"distinct_modes": len(n24), "columns": len(nd), "points": rd.numel(),
                                       "ms": t_dup, "values_per_s": od.numel() / (t_dup * 1e-3),
                                       "write_gbs": wbytes / (t_dup * 1e-3) / 1e9}
    del od
    return res


def measure_basis_latency(dev, steps: int = 200) -> dict:
    """basis_n20: 231 modes, 1000 points, R, R', R'' times the angular factor, plus d/dtheta Z."""
    import torch

    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import inputs

    cfg = inputs.WORKLOADS["basis_n20"]
    ns, ms = inputs.full_zernike_modes(cfg["n_max"])
    r, th = inputs.uniform_points(cfg["n_points"], cfg["seed"])
    plan = zp.Plan(ns, ms, device=dev)
    rt, tt = (torch.as_tensor(x, device=dev) for x in (r, th))
    stream = torch.cuda.current_stream(dev)
    fn = lambda: zp.basis(None, None, rt, tt, 2, dtheta=True, plan=plan)  # noqa: E731
    fn()
    ms_call = _events_ms(stream, fn, steps)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            fn()
    stream.wait_stream(side)
    g.replay()
    ms_graph = _events_ms(stream, g.replay, steps)
    vals = len(ns) * len(r) * 4
    return {"workload": "basis_n20", "modes": len(ns), "points": len(r), "us_per_call": ms_call * 1e3,
            "us_per_graph_replay": ms_graph * 1e3, "values_per_s_graph": vals / (ms_graph * 1e-3)}


def measure_batched(dev, steps: int = 3, n_instances: int = 512, point_scale: float = 1.0,
                    tune: bool = True) -> dict:
    """batched_512: 512 instances, n_max ~ U{8..64} (full Z sets), points log-uniform in
    [1e3, 2e5], 16 coefficient sets.  Persistent forward (float64 and float32 contraction) as a
    CUDA-graph replay after autotuning, the same float64 forward as one launch per instance,
    and the float64 adjoint (grad_r, grad_theta, grad_C)."""
    import torch

    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import inputs

    cfg = inputs.WORKLOADS["batched_512"]
    raw = inputs.batched_instances(n_instances, cfg["n_sets"], cfg["seed"], point_scale=point_scale)
    S = cfg["n_sets"]
    inst = []
    gen = torch.Generator(dev).manual_seed(5)
    for x in raw:
        inst.append({"n": x.n, "m": x.m, "r": torch.as_tensor(x.r, device=dev),
                     "theta": torch.as_tensor(x.theta, device=dev), "coeffs": torch.as_tensor(x.coeffs, device=dev),
                     "grad_out": torch.randn((len(x.r), S), dtype=torch.float64, device=dev, generator=gen)})
    points = sum(len(x.r) for x in raw)
    basis_values = sum(len(x.r) * len(x.n) for x in raw)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "batched_512", "instances": len(raw), "points": points, "sets": S,
           "basis_values": basis_values}
    b = zp.Batch(inst, S)
    cfg64 = b.tune("forward", "fp64", reps=1)[0] if tune else b.config()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            b.forward("fp64")
    stream.wait_stream(side)
    g.replay()
    t_graph = _events_ms(stream, g.replay, steps)
    t_per = _events_ms(stream, b.forward_per_instance, 1)
    cfg_adj = b.tune("adjoint", reps=1)[0] if tune else b.config()
    b.adjoint("fp64")
    t_adj = _events_ms(stream, lambda: b.adjoint("fp64"), 1)
    adj64 = [rec["grad_coeffs"].clone() for rec in b.instances]
    # The adjoint with the float64-accurate tensor-core contractions (per instance).
    b.adjoint("fp64emu")
    t_adj_emu = _events_ms(stream, lambda: b.adjoint("fp64emu"), 1)
    out["fp64emu_adjoint_ms"] = t_adj_emu
    out["fp64emu_adjoint_grad_coeffs_max_abs_diff_vs_fp64"] = max(
        float((rec["grad_coeffs"] - a).abs().max()) for rec, a in zip(b.instances, adj64) if a.numel())
    out["speedup_emulated_vs_fp64_adjoint"] = t_adj / t_adj_emu
    del adj64
    out["fp64_forward_graph_ms"] = t_graph
    out["fp64_forward_per_instance_launches_ms"] = t_per
    out["fp64_adjoint_ms"] = t_adj
    out["tuned_forward_cfg"] = list(cfg64)
    out["tuned_adjoint_cfg"] = list(cfg_adj)
    out["fp64_forward_basis_values_per_s"] = basis_values / (t_graph * 1e-3)
    # The fused float64-accurate forward on the tensor cores (basis generated inside the MMA
    # kernel), also as a CUDA-graph replay, against the float64 CUDA-core contraction above.
    ref = [rec["out"].clone() for rec in b.instances]
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g2, stream=side):
            b.forward("fp64emu")
    stream.wait_stream(side)
    g2.replay()
    t_fused = _events_ms(stream, g2.replay, steps)
    diff = max(float((rec["out"] - r0).abs().max()) for rec, r0 in zip(b.instances, ref) if r0.numel())
    mag = max(float(r0.abs().max()) for r0 in ref if r0.numel())
    out["fp64emu_fused_forward_graph_ms"] = t_fused
    out["fp64emu_fused_forward_basis_values_per_s"] = basis_values / (t_fused * 1e-3)
    out["fp64emu_fused_max_abs_diff_vs_fp64"] = diff
    out["fp64emu_fused_max_abs_value"] = mag
    out["speedup_fused_vs_fp64_forward"] = t_graph / t_fused
    del ref
    b.close()
    b32 = zp.Batch(inst, S, out_dtype=torch.float32, with_adjoint=False)
    cfg32 = b32.tune("forward", "fp32", reps=1)[0] if tune else b32.config()
    b32.forward("fp32")
    out["fp32_forward_ms"] = _events_ms(stream, lambda: b32.forward("fp32"), steps)
    out["tuned_fp32_cfg"] = list(cfg32)
    b32.close()
    return out


def measure_batched_adjoint(dev, steps: int = 2, n_instances: int = 512) -> dict:
    """batched_512's float64-accurate adjoint alone (one warm-up call, then `steps` timed calls):
    the two fused derivative-series passes and the per-instance grad_C."""
    import torch

    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import inputs

    cfg = inputs.WORKLOADS["batched_512"]
    raw = inputs.batched_instances(n_instances, cfg["n_sets"], cfg["seed"])
    S = cfg["n_sets"]
    gen = torch.Generator(dev).manual_seed(5)
    inst = [{"n": x.n, "m": x.m, "r": torch.as_tensor(x.r, device=dev), "theta": torch.as_tensor(x.theta, device=dev),
             "coeffs": torch.as_tensor(x.coeffs, device=dev),
             "grad_out": torch.randn((len(x.r), S), dtype=torch.float64, device=dev, generator=gen)} for x in raw]
    b = zp.Batch(inst, S)
    stream = torch.cuda.current_stream(dev)
    b.adjoint("fp64emu")
    t = _events_ms(stream, lambda: b.adjoint("fp64emu"), steps)
    b.close()
    return {"workload": "batched_512", "instances": len(raw), "points": sum(len(x.r) for x in raw), "sets": S,
            "fp64emu_adjoint_ms": t}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args) -> None:
    """The oracle as it stands on the host cores: each step is a bounded sample of the same
    workload (all modes, k = 0..3, a fixed set of points)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    n_pts = max(os.cpu_count() or 1, 16)
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.time(n_pts)
        vals = [pool.time(n_pts) for _ in range(args.steps)]
    finally:
        pool.close()
    value = statistics.mean(v["value"] for v in vals)
    ms_per_step = statistics.mean(1e3 * n_pts * 2601 * 4 / v["value"] for v in vals)
    cpu = dict(vals[0])
    cpu["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "exact rational (rounded to f64)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "modes": 2601, "n_max": 100, "points": 100_000, "derivs": 4,
                       "parallelism": "host cores", "sample_points_per_step": n_pts},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.batched_adjoint_only:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps({"batched_adjoint_only": measure_batched_adjoint(torch.device("cuda", 0), steps=args.steps,
                                                                          n_instances=args.batched_instances)}),
              flush=True)
        return
    if args.batched_only:
        import torch

        torch.cuda.set_device(0)
        res = measure_batched(torch.device("cuda", 0), steps=args.steps, n_instances=args.batched_instances,
                              point_scale=args.batched_point_scale, tune=False)
        print(json.dumps({"batched_only": res}), flush=True)
        return
    if args.fp64_probe_only:
        import ctypes

        import torch

        from paper_2409_19156_gb300 import _lib

        torch.cuda.set_device(0)
        lib = _lib.load()
        sp = torch.cuda.current_stream().cuda_stream
        out = []
        for op, name in ((0, "fma"), (1, "mul"), (2, "add")):
            for iters in (4000, 20000):
                res = (ctypes.c_double * 6)()
                _lib.check("zp_probe_fp64", lib.zp_probe_fp64(op, iters, sp, res))
                out.append({"op": name, "iters": iters, "ops_per_s": res[2], "lanes_per_sm_clk": res[3],
                            "implied_sm_mhz": res[4], "ms": res[1]})
        print(json.dumps({"fp64_probe_only": out}), flush=True)
        return
    if args.fused_only:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps({"fused_only": measure_fused_series(torch.device("cuda", 0), {}, steps=args.steps,
                                                             n_points=args.fused_points)}), flush=True)
        return
    if args.adjoint_emulated_only:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps({"adjoint_emulated_only": measure_adjoint_emulated(torch.device("cuda", 0),
                                                                            steps=args.steps)}), flush=True)
        return
    if args.paper_shapes_only:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps({"paper_shapes_only": measure_paper_shapes(torch.device("cuda", 0), steps=args.steps)}),
              flush=True)
        return
    if args.adjoint_only:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps({"adjoint_only": measure_adjoint(torch.device("cuda", 0), steps=args.steps)}), flush=True)
        return
    if args.series_only:
        import torch

        torch.cuda.set_device(0)
        res = measure_series(torch.device("cuda", 0), {}, steps=args.steps, n_points=args.series_points,
                             with_fp64=False, with_emulated_only=args.series_emulated, n_sets=args.series_sets)
        print(json.dumps({"series_only": res}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
