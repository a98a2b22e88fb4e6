// Series of Zernike functions and its adjoint, float64.
//
//   F = Z^T C                     (Z: basis [J][P] written by the walk kernel to scratch)
//   grad_C = Z G                  (float64-accurate tensor-core GEMM of zp_mma.cu by default;
//                                  cuBLAS DGEMM for ZP_PREC_FP64, the plain baseline form)
//   H = C G^T  -> [J][P]          (the same, point-fastest so the next kernel coalesces)
//   grad_r[p]     = sum_j dZ_j/drho(p)   H[j][p]
//   grad_theta[p] = sum_j dZ_j/dtheta(p) H[j][p]
// The last two are one kernel that regenerates the basis derivatives in registers (the
// per-column recursion of zp_walk.cu with one rho-derivative lane) and reduces over all
// modes inside one thread per point: no partial buffers, no atomics, deterministic.
// Scratch is allocated stream-ordered (cudaMallocAsync) and released on the same stream.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "zp_device.cuh"
#include "zp_api_common.h"
#include "zp_fused.h"
#include "zp_series_internal.h"

namespace zp {
namespace {

constexpr int kRedThreads = 128;

// One thread per point: walks every |m| column (Taylor lanes k <= 1, or k <= 2 with HESS) and
// accumulates, with H[j][p] = sum_s C[j, s] G[p, s],
//   grad_r  = sum_j dZ_j/drho H,        grad_theta = sum_j dZ_j/dtheta H,
//   and with HESS the point's 2x2 Hessian block of L = <G, F>:
//   hess_rr = sum_j d2Z_j/drho2 H,  hess_rt = sum_j d2Z_j/drho dtheta H,  hess_tt = sum_j d2Z_j/dtheta2 H,
//   and, given a tangent (v_r, v_theta), the Hessian-vector product
//   hv_r = hess_rr v_r + hess_rt v_theta,  hv_theta = hess_rt v_r + hess_tt v_theta.
// (The Hessian of L in the point coordinates is block diagonal: r_p and theta_p only enter row p.)

template <bool HESS>
__global__ void __launch_bounds__(kRedThreads)
adjoint_point_kernel(const Column* __restrict__ cols, int n_cols, const double* __restrict__ table,
                     const int32_t* __restrict__ slot_ptr, const int32_t* __restrict__ slot_idx,
                     const double* __restrict__ r, const double* __restrict__ theta, int64_t P,
                     const double* __restrict__ H, double* grad_r, double* grad_theta, HessOut ho) {
  const int64_t p = (int64_t)blockIdx.x * kRedThreads + threadIdx.x;
  if (p >= P) return;
  const double rho = r[p], u = rho * rho, th = theta[p];
  double acc_r = 0.0, acc_t = 0.0, acc_rr = 0.0, acc_rt = 0.0, acc_tt = 0.0;
  // cos / sin(m theta) and rho^(m-2), rho^(m-1), rho^m: advanced by one angle addition and one
  // product when the next column has m + 1 (the usual column order), else computed directly.
  double s1, c1;
  sincos(th, &s1, &c1);
  double cs = 1.0, sn = 0.0, pm2 = 0.0, pm1 = 0.0, pm = 1.0;
  int m_prev = 0;
  for (int c = 0; c < n_cols; ++c) {
    const Column col = cols[c];
    const int m = col.m;
    const double* h = table + (size_t)col.table_row * kRow;
    const int32_t* sp = slot_ptr + col.slot_base;
    if (c > 0 && m == m_prev + 1) {
      const double cn = fma(cs, c1, -sn * s1);
      sn = fma(sn, c1, cs * s1);
      cs = cn;
      pm2 = pm1;
      pm1 = pm;
      pm *= rho;
    } else if (c == 0 || m != m_prev) {
      cs = 1.0;
      sn = 0.0;
      if (m != 0) sincos((double)m * th, &sn, &cs);
      // Seeds of the Taylor lanes: N = 0 -> rho^m, N = 1 -> (m+2) rho^(m+2) - (m+1) rho^m.
      pm2 = m >= 2 ? pow_uint(rho, m - 2) : 0.0;
      pm1 = m >= 2 ? pm2 * rho : (m == 1 ? 1.0 : 0.0);
      pm = m >= 1 ? pm1 * rho : 1.0;
    }
    m_prev = m;
    double T0 = pm, T1 = h[1] * pm1, T2 = HESS ? h[2] * pm2 : 0.0;
    double S0 = fma(h[4], pm * u, -(h[8] * pm));
    double S1 = fma(h[5], pm * rho, -(h[9] * pm1));
    double S2 = HESS ? fma(h[6], pm, -(h[10] * pm2)) : 0.0;
    const double md = (double)m;
    auto accumulate = [&](int N, double v0, double v1, double v2) {
      const int sb = sp[N], se = sp[N + 1];
      if (sb == se) return;
      const double* row = h + (size_t)(kHeaderRows + N) * kRow;
      const double zero = row[7];  // 0.0: products issue as DFMA, faster than DMUL on GB300
      const double R0 = fma(row[3], v0, zero), R1 = fma(row[4], v1, zero);
      const double R2 = HESS ? fma(row[5], v2, zero) : 0.0;
      for (int s = sb; s < se; ++s) {
        const uint32_t code = (uint32_t)__ldg(slot_idx + s);
        const int64_t j = (int64_t)(code & 0x7fffffffu);
        const bool is_sin = (code >> 31) != 0;
        const double hv = H[j * P + p];
        const double f = is_sin ? sn : cs;
        const double dt = is_sin ? md * cs : -md * sn;
        acc_r = fma(fma(R1, f, zero), hv, acc_r);
        acc_t = fma(fma(R0, dt, zero), hv, acc_t);
        if constexpr (HESS) {
          acc_rr = fma(fma(R2, f, zero), hv, acc_rr);
          acc_rt = fma(fma(R1, dt, zero), hv, acc_rt);
          acc_tt = fma(fma(R0, -md * md * f, zero), hv, acc_tt);
        }
      }
    };
    accumulate(0, T0, T1, T2);
    if (col.n_steps < 2) continue;
    accumulate(1, S0, S1, S2);
    for (int N = 2; N < col.n_steps; ++N) {
      const double* row = h + (size_t)(kHeaderRows + N) * kRow;
      const double A = row[0], B = row[1], A2 = row[2];
      const double g = fma(A, u, -B);
      const double hg = fma(A2, rho, row[7]);
      const double n0 = fma(g, S0, -T0);
      const double n1 = fma(g, S1, fma(hg, S0, -T1));
      if constexpr (HESS) {
        const double n2 = fma(g, S2, fma(hg, S1, fma(A, S0, -T2)));
        T2 = S2;
        S2 = n2;
      }
      T0 = S0;
      T1 = S1;
      S0 = n0;
      S1 = n1;
      accumulate(N, S0, S1, S2);
    }
  }
  if (grad_r) grad_r[p] = acc_r;
  if (grad_theta) grad_theta[p] = acc_t;
  if constexpr (HESS) {
    if (ho.rr) ho.rr[p] = acc_rr;
    if (ho.rt) ho.rt[p] = acc_rt;
    if (ho.tt) ho.tt[p] = acc_tt;
    if (ho.v_r) {
      const double vr = ho.v_r[p], vt = ho.v_theta[p];
      if (ho.hv_r) ho.hv_r[p] = fma(acc_rr, vr, acc_rt * vt);
      if (ho.hv_theta) ho.hv_theta[p] = fma(acc_rt, vr, acc_tt * vt);
    }
  }
}

struct CublasHandles {
  std::mutex mu;
  std::vector<cublasHandle_t> per_device;
};

CublasHandles& handles() {
  static CublasHandles h;
  return h;
}

const char* cublas_name(cublasStatus_t s) {
  switch (s) {
    case CUBLAS_STATUS_SUCCESS: return "CUBLAS_STATUS_SUCCESS";
    case CUBLAS_STATUS_NOT_INITIALIZED: return "CUBLAS_STATUS_NOT_INITIALIZED";
    case CUBLAS_STATUS_ALLOC_FAILED: return "CUBLAS_STATUS_ALLOC_FAILED";
    case CUBLAS_STATUS_INVALID_VALUE: return "CUBLAS_STATUS_INVALID_VALUE";
    case CUBLAS_STATUS_ARCH_MISMATCH: return "CUBLAS_STATUS_ARCH_MISMATCH";
    case CUBLAS_STATUS_EXECUTION_FAILED: return "CUBLAS_STATUS_EXECUTION_FAILED";
    case CUBLAS_STATUS_NOT_SUPPORTED: return "CUBLAS_STATUS_NOT_SUPPORTED";
    default: return "CUBLAS_STATUS_OTHER";
  }
}

}  // namespace

// Thread-safe: one handle per device, serialised by the lock for the duration of a call
// sequence (set-stream + gemm) through the Lock object.
struct CublasLock {
  std::unique_lock<std::mutex> lock;
  cublasHandle_t h = nullptr;
};

static zp_status get_cublas(CublasLock& out, cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  CublasHandles& hs = handles();
  out.lock = std::unique_lock<std::mutex>(hs.mu);
  if ((int)hs.per_device.size() <= dev) hs.per_device.resize(dev + 1, nullptr);
  if (!hs.per_device[dev]) {
    cublasStatus_t s = cublasCreate(&hs.per_device[dev]);
    if (s != CUBLAS_STATUS_SUCCESS) return set_error(ZP_ERR_CUDA, std::string("cublasCreate: ") + cublas_name(s));
  }
  out.h = hs.per_device[dev];
  cublasStatus_t s = cublasSetStream(out.h, stream);
  if (s != CUBLAS_STATUS_SUCCESS) return set_error(ZP_ERR_CUDA, std::string("cublasSetStream: ") + cublas_name(s));
  return ZP_OK;
}

// Column-major DGEMM wrapper: C = op(A) op(B).
static zp_status dgemm(cublasHandle_t h, bool ta, bool tb, int64_t m, int64_t n, int64_t k, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc) {
  const double one = 1.0, zero = 0.0;
  cublasStatus_t s = cublasDgemm_64(h, ta ? CUBLAS_OP_T : CUBLAS_OP_N, tb ? CUBLAS_OP_T : CUBLAS_OP_N, m, n, k, &one,
                                    A, lda, B, ldb, &zero, C, ldc);
  if (s != CUBLAS_STATUS_SUCCESS) return set_error(ZP_ERR_CUDA, std::string("cublasDgemm: ") + cublas_name(s));
  return ZP_OK;
}

// The library's own stream-ordered memory pool per device.  Up to kScratchKeepBytes of freed
// scratch stay reserved across synchronisations: the default pool hands freed memory back at
// every synchronisation, and mapping it again cost 0.7-1.2 ms of host time per call (the
// emulated float64 series and adjoint, and every fit, which synchronises).
constexpr uint64_t kScratchKeepBytes = 16ull << 30;
struct ScratchPools {
  std::mutex mu;
  cudaMemPool_t pool[64] = {};
};
ScratchPools& scratch_pools() {
  static ScratchPools p;
  return p;
}
zp_status scratch_pool(cudaMemPool_t* out, bool create) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(ZP_ERR_UNSUPPORTED, "device ordinal above 63");
  ScratchPools& ps = scratch_pools();
  std::lock_guard<std::mutex> lock(ps.mu);
  if (!ps.pool[dev] && create) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return cuda_error(e, "cudaMemPoolCreate");
    uint64_t keep = kScratchKeepBytes;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return cuda_error(e, "cudaMemPoolSetAttribute");
    }
    ps.pool[dev] = pool;
  }
  *out = ps.pool[dev];
  return ZP_OK;
}

ScratchBuffer::~ScratchBuffer() {
  if (ptr) cudaFreeAsync(ptr, stream);
}

zp_status ScratchBuffer::alloc(size_t bytes, cudaStream_t s) {
  stream = s;
  if (bytes == 0) return ZP_OK;
  cudaMemPool_t pool = nullptr;
  ZP_TRY(scratch_pool(&pool, true));
  cudaError_t e = cudaMallocFromPoolAsync(&ptr, bytes, pool, s);
  if (e != cudaSuccess) {
    ptr = nullptr;
    return cuda_error(e, "cudaMallocFromPoolAsync(scratch)");
  }
  return ZP_OK;
}

zp_status series_eval_fp64(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                           const double* coeffs, int64_t S, double* out, cudaStream_t stream) {
  const int64_t J = plan->n_modes;
  ScratchBuffer z;
  ZP_TRY(z.alloc((size_t)J * P * sizeof(double), stream));
  ZP_TRY(launch_walk(plan, r, theta, P, 0, (double*)z.ptr, nullptr, stream));
  CublasLock cl;
  ZP_TRY(get_cublas(cl, stream));
  // F (row-major [P][S]) = column-major S x P = C^T(S x J) * Z(J x P):
  //   C row-major [J][S] is column-major S x J (ld S); Z row-major [J][P] is column-major P x J -> op T.
  return dgemm(cl.h, false, true, S, P, J, coeffs, S, (const double*)z.ptr, P, out, S);
}

zp_status series_adjoint_fp64(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                              const double* coeffs, int64_t S, const double* G, double* grad_coeffs, double* grad_r,
                              double* grad_theta, cudaStream_t stream, const HessOut& ho, bool emulated) {
  const int64_t J = plan->n_modes;
  // Few sets, emulated, no Hessian: the point gradients come from the fused kernel's
  // derivative series (no [modes x points] H).
  const bool fused_pt = emulated && !ho.any() && (grad_r || grad_theta) && S <= kFusedMaxSets &&
                        plan->fused_kpad <= kFusedMaxModes;
  if (fused_pt) ZP_TRY(fused_point_grads(plan, r, theta, P, coeffs, S, G, grad_r, grad_theta, stream));
  const bool need_h = !fused_pt && (grad_r || grad_theta || ho.any());
  ScratchBuffer z, hbuf;
  CublasLock cl;
  if (grad_coeffs) {
    ZP_TRY(z.alloc((size_t)J * P * sizeof(double), stream));
    if (emulated) {
      // grad_C[j][s] = sum_p Z[j][p] G[p][s]: A(j, p) = Z[j * P + p], B(s, p) = G[p * S + s];
      // the walk also forms Z's row maxima for A's row scales.
      ScratchBuffer zmax;
      ZP_TRY(zmax.alloc((size_t)J * sizeof(unsigned long long), stream));
      const cudaError_t e = cudaMemsetAsync(zmax.ptr, 0, (size_t)J * sizeof(unsigned long long), stream);
      if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
      ZP_TRY(launch_walk(plan, r, theta, P, 0, (double*)z.ptr, nullptr, stream, nullptr,
                         (unsigned long long*)zmax.ptr));
      ZP_TRY(emulated_gemm_fp64(J, S, P, (const double*)z.ptr, P, 1, G, 1, S, grad_coeffs, S, stream,
                                (const unsigned long long*)zmax.ptr));
    } else {
      ZP_TRY(launch_walk(plan, r, theta, P, 0, (double*)z.ptr, nullptr, stream));
      ZP_TRY(get_cublas(cl, stream));
      // grad_C row-major [J][S] = column-major S x J = G^T (S x P) * Z^T (P x J):
      //   G row-major [P][S] is column-major S x P; Z row-major [J][P] is column-major P x J.
      ZP_TRY(dgemm(cl.h, false, false, S, J, P, G, S, (const double*)z.ptr, P, grad_coeffs, S));
    }
  }
  if (need_h) {
    ZP_TRY(hbuf.alloc((size_t)J * P * sizeof(double), stream));
    if (emulated) {
      // H[j][p] = sum_s C[j][s] G[p][s]: A(j, s) = C[j * S + s], B(p, s) = G[p * S + s].
      ZP_TRY(emulated_gemm_fp64(J, P, S, coeffs, S, 1, G, S, 1, (double*)hbuf.ptr, P, stream));
    } else {
      if (!cl.h) ZP_TRY(get_cublas(cl, stream));
      // H row-major [J][P] = column-major P x J = G (P x S) * C^T (S x J):
      //   G column-major S x P -> op T; C column-major S x J -> op N.
      ZP_TRY(dgemm(cl.h, true, false, P, J, S, G, S, coeffs, S, (double*)hbuf.ptr, P));
    }
    const int64_t blocks = (P + kRedThreads - 1) / kRedThreads;
    if (ho.any())
      adjoint_point_kernel<true><<<(unsigned)blocks, kRedThreads, 0, stream>>>(
          plan->dev.cols, (int)plan->cols.size(), plan->dev.table, plan->dev.slot_ptr, plan->dev.slot_idx, r, theta, P,
          (const double*)hbuf.ptr, grad_r, grad_theta, ho);
    else
      adjoint_point_kernel<false><<<(unsigned)blocks, kRedThreads, 0, stream>>>(
          plan->dev.cols, (int)plan->cols.size(), plan->dev.table, plan->dev.slot_ptr, plan->dev.slot_idx, r, theta, P,
          (const double*)hbuf.ptr, grad_r, grad_theta, HessOut());
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "adjoint_point_kernel launch");
  }
  return ZP_OK;
}

}  // namespace zp

using namespace zp;

static zp_status series_args(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                             const double* coeffs, int64_t S) {
  ZP_TRY(check_plan_device(plan));
  if (P < 0) return set_error(ZP_ERR_INVALID_ARG, "n_points < 0");
  if (S < 0) return set_error(ZP_ERR_INVALID_ARG, "n_sets < 0");
  if (P == 0 || plan->n_modes == 0 || S == 0) return ZP_OK;
  ZP_TRY(check_device_array(r, "r", 8));
  ZP_TRY(check_device_array(theta, "theta", 8));
  ZP_TRY(check_device_array(coeffs, "coeffs", 8));
  return ZP_OK;
}

extern "C" {

static zp_status zp_series_eval_plan_impl(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                              const double* coeffs, int64_t n_sets, zp_precision prec, void* out, void* stream) {
  clear_error();
  if (prec != ZP_PREC_FP64 && prec != ZP_PREC_BF16X3 && prec != ZP_PREC_TF32 && prec != ZP_PREC_FP64_EMULATED)
    return set_error(ZP_ERR_INVALID_ARG, "unknown precision for zp_series_eval");
  const bool f64_out = prec == ZP_PREC_FP64 || prec == ZP_PREC_FP64_EMULATED;
  ZP_TRY(series_args(plan, r, theta, n_points, coeffs, n_sets));
  if (n_points == 0 || n_sets == 0) return ZP_OK;
  ZP_TRY(check_device_array(out, "out", f64_out ? 8 : 16));
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->n_modes == 0) {
    const size_t bytes = (size_t)n_points * n_sets * (f64_out ? 8 : 4);
    cudaError_t e = cudaMemsetAsync(out, 0, bytes, st);
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "cudaMemsetAsync");
  }
  if (prec == ZP_PREC_FP64) return series_eval_fp64(plan, r, theta, n_points, coeffs, n_sets, (double*)out, st);
  if (prec == ZP_PREC_FP64_EMULATED) {
    // Few sets: the fused kernel (basis generated on chip, no basis or partial sums in HBM).
    if (n_sets <= kFusedMaxSets && plan->fused_kpad <= kFusedMaxModes)
      return fused_series_eval(plan, r, theta, n_points, coeffs, n_sets, (double*)out, st);
    return series_eval_emulated_fp64(plan, r, theta, n_points, coeffs, n_sets, (double*)out, st);
  }
  return series_eval_split(plan, r, theta, n_points, coeffs, n_sets, prec, (float*)out, st);
}

zp_status zp_series_eval_plan(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                              const double* coeffs, int64_t n_sets, zp_precision prec, void* out, void* stream) {
  zp::NvtxRange zp_range_("zp_series_eval_plan");
  return zp::entry_finish("zp_series_eval_plan", stream, zp_series_eval_plan_impl(plan, r, theta, n_points, coeffs, n_sets, prec, out, stream));
}

zp_status zp_series_eval_timed(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                               const double* coeffs, int64_t n_sets, zp_precision prec, void* out, void* stream,
                               float* phase_ms) {
  clear_error();
  if (!phase_ms) return set_error(ZP_ERR_INVALID_ARG, "phase_ms is NULL");
  if (prec != ZP_PREC_BF16X3 && prec != ZP_PREC_TF32)
    return set_error(ZP_ERR_INVALID_ARG, "timed series supports the split precisions only");
  ZP_TRY(series_args(plan, r, theta, n_points, coeffs, n_sets));
  phase_ms[0] = phase_ms[1] = phase_ms[2] = 0.0f;
  if (n_points == 0 || n_sets == 0 || plan->n_modes == 0) return ZP_OK;
  ZP_TRY(check_device_array(out, "out", 16));
  return series_eval_split(plan, r, theta, n_points, coeffs, n_sets, prec, (float*)out, (cudaStream_t)stream,
                           phase_ms);
}

static zp_status zp_series_eval_impl(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r, const double* theta,
                         int64_t n_points, const double* coeffs, int64_t n_sets, zp_precision prec, void* out,
                         void* stream) {
  clear_error();
  std::shared_ptr<const zp_plan> held;
  ZP_TRY(cached_plan(n, m, n_modes, &held));
  const zp_plan* plan = held.get();
  return zp_series_eval_plan(plan, r, theta, n_points, coeffs, n_sets, prec, out, stream);
}

zp_status zp_series_eval(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r, const double* theta,
                         int64_t n_points, const double* coeffs, int64_t n_sets, zp_precision prec, void* out,
                         void* stream) {
  zp::NvtxRange zp_range_("zp_series_eval");
  return zp::entry_finish("zp_series_eval", stream, zp_series_eval_impl(n, m, n_modes, r, theta, n_points, coeffs, n_sets, prec, out, stream));
}

static zp_status zp_series_adjoint_plan_impl(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                                 const double* coeffs, int64_t n_sets, const double* grad_out, double* grad_coeffs,
                                 double* grad_r, double* grad_theta, void* stream) {
  return zp_series_adjoint_plan_prec(plan, r, theta, n_points, coeffs, n_sets, grad_out, grad_coeffs, grad_r,
                                     grad_theta, ZP_PREC_FP64_EMULATED, stream);
}

zp_status zp_series_adjoint_plan(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                                 const double* coeffs, int64_t n_sets, const double* grad_out, double* grad_coeffs,
                                 double* grad_r, double* grad_theta, void* stream) {
  zp::NvtxRange zp_range_("zp_series_adjoint_plan");
  return zp::entry_finish("zp_series_adjoint_plan", stream, zp_series_adjoint_plan_impl(plan, r, theta, n_points, coeffs, n_sets, grad_out, grad_coeffs, grad_r, grad_theta, stream));
}

static zp_status zp_series_adjoint_plan_prec_impl(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                                      const double* coeffs, int64_t n_sets, const double* grad_out,
                                      double* grad_coeffs, double* grad_r, double* grad_theta, zp_precision prec,
                                      void* stream) {
  clear_error();
  if (prec != ZP_PREC_FP64 && prec != ZP_PREC_FP64_EMULATED)
    return set_error(ZP_ERR_INVALID_ARG, "the adjoint takes ZP_PREC_FP64 or ZP_PREC_FP64_EMULATED");
  ZP_TRY(series_args(plan, r, theta, n_points, coeffs, n_sets));
  if (grad_coeffs) ZP_TRY(check_device_array(grad_coeffs, "grad_coeffs", 8));
  if (grad_r) ZP_TRY(check_device_array(grad_r, "grad_r", 8));
  if (grad_theta) ZP_TRY(check_device_array(grad_theta, "grad_theta", 8));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t J = plan->n_modes, P = n_points, S = n_sets;
  if (P == 0 || J == 0 || S == 0) {
    // Empty sums: zero whatever gradient exists.
    cudaError_t e = cudaSuccess;
    if (grad_coeffs && J * S > 0) e = cudaMemsetAsync(grad_coeffs, 0, (size_t)J * S * 8, st);
    if (e == cudaSuccess && grad_r && P > 0) e = cudaMemsetAsync(grad_r, 0, (size_t)P * 8, st);
    if (e == cudaSuccess && grad_theta && P > 0) e = cudaMemsetAsync(grad_theta, 0, (size_t)P * 8, st);
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "cudaMemsetAsync");
  }
  ZP_TRY(check_device_array(grad_out, "grad_out", 8));
  return series_adjoint_fp64(plan, r, theta, P, coeffs, S, grad_out, grad_coeffs, grad_r, grad_theta, st, HessOut(),
                             prec == ZP_PREC_FP64_EMULATED);
}

zp_status zp_series_adjoint_plan_prec(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                                      const double* coeffs, int64_t n_sets, const double* grad_out,
                                      double* grad_coeffs, double* grad_r, double* grad_theta, zp_precision prec,
                                      void* stream) {
  zp::NvtxRange zp_range_("zp_series_adjoint_plan_prec");
  return zp::entry_finish("zp_series_adjoint_plan_prec", stream, zp_series_adjoint_plan_prec_impl(plan, r, theta, n_points, coeffs, n_sets, grad_out, grad_coeffs, grad_r, grad_theta, prec, stream));
}

static zp_status zp_series_point_hessian_plan_impl(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                                       const double* coeffs, int64_t n_sets, const double* grad_out, double* grad_r,
                                       double* grad_theta, double* hess_rr, double* hess_rt, double* hess_tt,
                                       void* stream) {
  clear_error();
  ZP_TRY(series_args(plan, r, theta, n_points, coeffs, n_sets));
  double* outs[5] = {grad_r, grad_theta, hess_rr, hess_rt, hess_tt};
  const char* names[5] = {"grad_r", "grad_theta", "hess_rr", "hess_rt", "hess_tt"};
  for (int i = 0; i < 5; ++i)
    if (outs[i]) ZP_TRY(check_device_array(outs[i], names[i], 8));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t J = plan->n_modes, P = n_points, S = n_sets;
  if (P == 0) return ZP_OK;
  if (J == 0 || S == 0) {
    for (int i = 0; i < 5; ++i) {
      if (!outs[i]) continue;
      cudaError_t e = cudaMemsetAsync(outs[i], 0, (size_t)P * 8, st);
      if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
    }
    return ZP_OK;
  }
  ZP_TRY(check_device_array(grad_out, "grad_out", 8));
  HessOut ho;
  ho.rr = hess_rr;
  ho.rt = hess_rt;
  ho.tt = hess_tt;
  return series_adjoint_fp64(plan, r, theta, P, coeffs, S, grad_out, nullptr, grad_r, grad_theta, st, ho,
                             /*emulated=*/true);
}

zp_status zp_series_point_hessian_plan(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                                       const double* coeffs, int64_t n_sets, const double* grad_out, double* grad_r,
                                       double* grad_theta, double* hess_rr, double* hess_rt, double* hess_tt,
                                       void* stream) {
  zp::NvtxRange zp_range_("zp_series_point_hessian_plan");
  return zp::entry_finish("zp_series_point_hessian_plan", stream, zp_series_point_hessian_plan_impl(plan, r, theta, n_points, coeffs, n_sets, grad_out, grad_r, grad_theta, hess_rr, hess_rt, hess_tt, stream));
}

static zp_status zp_series_point_hvp_plan_impl(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                                   const double* coeffs, int64_t n_sets, const double* grad_out, const double* v_r,
                                   const double* v_theta, double* hv_r, double* hv_theta, void* stream) {
  clear_error();
  ZP_TRY(series_args(plan, r, theta, n_points, coeffs, n_sets));
  if (hv_r) ZP_TRY(check_device_array(hv_r, "hv_r", 8));
  if (hv_theta) ZP_TRY(check_device_array(hv_theta, "hv_theta", 8));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t J = plan->n_modes, P = n_points, S = n_sets;
  if (P == 0 || (!hv_r && !hv_theta)) return ZP_OK;
  if (J == 0 || S == 0) {
    cudaError_t e = cudaSuccess;
    if (hv_r) e = cudaMemsetAsync(hv_r, 0, (size_t)P * 8, st);
    if (e == cudaSuccess && hv_theta) e = cudaMemsetAsync(hv_theta, 0, (size_t)P * 8, st);
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "cudaMemsetAsync");
  }
  ZP_TRY(check_device_array(grad_out, "grad_out", 8));
  ZP_TRY(check_device_array(v_r, "v_r", 8));
  ZP_TRY(check_device_array(v_theta, "v_theta", 8));
  HessOut ho;
  ho.v_r = v_r;
  ho.v_theta = v_theta;
  ho.hv_r = hv_r;
  ho.hv_theta = hv_theta;
  return series_adjoint_fp64(plan, r, theta, P, coeffs, S, grad_out, nullptr, nullptr, nullptr, st, ho,
                             /*emulated=*/true);
}

zp_status zp_series_point_hvp_plan(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                                   const double* coeffs, int64_t n_sets, const double* grad_out, const double* v_r,
                                   const double* v_theta, double* hv_r, double* hv_theta, void* stream) {
  zp::NvtxRange zp_range_("zp_series_point_hvp_plan");
  return zp::entry_finish("zp_series_point_hvp_plan", stream, zp_series_point_hvp_plan_impl(plan, r, theta, n_points, coeffs, n_sets, grad_out, v_r, v_theta, hv_r, hv_theta, stream));
}

static zp_status zp_series_point_hessian_impl(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r,
                                  const double* theta, int64_t n_points, const double* coeffs, int64_t n_sets,
                                  const double* grad_out, double* grad_r, double* grad_theta, double* hess_rr,
                                  double* hess_rt, double* hess_tt, void* stream) {
  clear_error();
  std::shared_ptr<const zp_plan> held;
  ZP_TRY(cached_plan(n, m, n_modes, &held));
  const zp_plan* plan = held.get();
  return zp_series_point_hessian_plan(plan, r, theta, n_points, coeffs, n_sets, grad_out, grad_r, grad_theta, hess_rr,
                                      hess_rt, hess_tt, stream);
}

zp_status zp_series_point_hessian(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r,
                                  const double* theta, int64_t n_points, const double* coeffs, int64_t n_sets,
                                  const double* grad_out, double* grad_r, double* grad_theta, double* hess_rr,
                                  double* hess_rt, double* hess_tt, void* stream) {
  zp::NvtxRange zp_range_("zp_series_point_hessian");
  return zp::entry_finish("zp_series_point_hessian", stream, zp_series_point_hessian_impl(n, m, n_modes, r, theta, n_points, coeffs, n_sets, grad_out, grad_r, grad_theta, hess_rr, hess_rt, hess_tt, stream));
}

static zp_status zp_series_adjoint_impl(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r,
                            const double* theta, int64_t n_points, const double* coeffs, int64_t n_sets,
                            const double* grad_out, double* grad_coeffs, double* grad_r, double* grad_theta,
                            void* stream) {
  clear_error();
  std::shared_ptr<const zp_plan> held;
  ZP_TRY(cached_plan(n, m, n_modes, &held));
  const zp_plan* plan = held.get();
  return zp_series_adjoint_plan(plan, r, theta, n_points, coeffs, n_sets, grad_out, grad_coeffs, grad_r, grad_theta,
                                stream);
}

zp_status zp_series_adjoint(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r,
                            const double* theta, int64_t n_points, const double* coeffs, int64_t n_sets,
                            const double* grad_out, double* grad_coeffs, double* grad_r, double* grad_theta,
                            void* stream) {
  zp::NvtxRange zp_range_("zp_series_adjoint");
  return zp::entry_finish("zp_series_adjoint", stream, zp_series_adjoint_impl(n, m, n_modes, r, theta, n_points, coeffs, n_sets, grad_out, grad_coeffs, grad_r, grad_theta, stream));
}

}  // extern "C"

extern "C" ZP_API zp_status zp_release_scratch(void) {
  zp::clear_error();
  cudaMemPool_t pool = nullptr;
  ZP_TRY(zp::scratch_pool(&pool, false));
  if (!pool) return ZP_OK;
  const cudaError_t e = cudaMemPoolTrimTo(pool, 0);
  return e == cudaSuccess ? ZP_OK : zp::cuda_error(e, "cudaMemPoolTrimTo");
}
