// Least-squares fit of Zernike series coefficients (the "fit" counterpart of zp_series_eval).
//
//   minimise  sum_p w_p || sum_j Z_j(p) C[j, :] - Y[p, :] ||^2  +  ridge ||C||^2
//   =>  (Z W Z^T + ridge I) C = Z W Y          (normal equations, Z = basis [J][P])
//
// Steps: the basis by the walk kernel (float64, into scratch), the rows scaled by sqrt(w) when
// weights are given, the Gram matrix and the right-hand side by cuBLAS DGEMM (or by the
// float64-accurate tensor-core GEMM of zp_mma.cu for ZP_PREC_FP64_EMULATED), the
// ridge added on the diagonal, a Cholesky factorisation and solve by cuSOLVER, and a DGEAM
// transpose into the caller's row-major [J][S] output.  The call synchronises its stream at
// the end to read the factorisation status.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "zp_api_common.h"
#include "zp_series_internal.h"

namespace zp {
namespace {

// Z[j][p] *= sqrt(w[p]); Ys[p][s] = sqrt(w[p]) * Y[p][s].
__global__ void scale_rows_kernel(double* Z, int64_t J, int64_t P, const double* w) {
  const int64_t n = J * P;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Z[i] *= sqrt(w[i % P]);
}
__global__ void scale_samples_kernel(const double* Y, double* Ys, int64_t P, int64_t S, const double* w) {
  const int64_t n = P * S;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Ys[i] = Y[i] * sqrt(w[i / S]);
}
__global__ void add_ridge_kernel(double* G, int64_t J, double ridge) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J; i += (int64_t)gridDim.x * blockDim.x)
    G[i * J + i] += ridge;
}

// Smallest and largest squared pivot of the Cholesky factor (single block).
__global__ void pivot_range_kernel(const double* L, int64_t J, double* out) {
  __shared__ double smin[256], smax[256];
  double lo = 1.0 / 0.0, hi = 0.0;
  for (int64_t i = threadIdx.x; i < J; i += blockDim.x) {
    const double d = L[i * J + i];
    const double d2 = d * d;
    lo = d2 < lo ? d2 : lo;
    hi = d2 > hi ? d2 : hi;
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      smin[threadIdx.x] = smin[threadIdx.x + s] < smin[threadIdx.x] ? smin[threadIdx.x + s] : smin[threadIdx.x];
      smax[threadIdx.x] = smax[threadIdx.x + s] > smax[threadIdx.x] ? smax[threadIdx.x + s] : smax[threadIdx.x];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = smin[0];
    out[1] = smax[0];
  }
}

struct SolverHandles {
  std::mutex mu;
  std::vector<cusolverDnHandle_t> solver;
  std::vector<cublasHandle_t> blas;
};
SolverHandles& solver_handles() {
  static SolverHandles h;
  return h;
}

}  // namespace

zp_status series_fit_fp64(const zp_plan* plan, const double* r, const double* theta, const double* w, int64_t P,
                          const double* Y, int64_t S, double ridge, double* coeffs, cudaStream_t stream,
                          bool emulated) {
  const int64_t J = plan->n_modes;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  SolverHandles& hs = solver_handles();
  std::lock_guard<std::mutex> lock(hs.mu);
  if ((int)hs.solver.size() <= dev) {
    hs.solver.resize(dev + 1, nullptr);
    hs.blas.resize(dev + 1, nullptr);
  }
  if (!hs.solver[dev] && cusolverDnCreate(&hs.solver[dev]) != CUSOLVER_STATUS_SUCCESS)
    return set_error(ZP_ERR_CUDA, "cusolverDnCreate failed");
  if (!hs.blas[dev] && cublasCreate(&hs.blas[dev]) != CUBLAS_STATUS_SUCCESS)
    return set_error(ZP_ERR_CUDA, "cublasCreate failed");
  cusolverDnHandle_t sol = hs.solver[dev];
  cublasHandle_t blas = hs.blas[dev];
  if (cusolverDnSetStream(sol, stream) != CUSOLVER_STATUS_SUCCESS || cublasSetStream(blas, stream) != CUBLAS_STATUS_SUCCESS)
    return set_error(ZP_ERR_CUDA, "setting the stream of the solver handles failed");

  ScratchBuffer zbuf, ybuf, gram, rhs, info;
  ZP_TRY(zbuf.alloc((size_t)J * P * sizeof(double), stream));
  ZP_TRY(gram.alloc((size_t)J * J * sizeof(double), stream));
  ZP_TRY(rhs.alloc((size_t)J * S * sizeof(double), stream));
  ZP_TRY(info.alloc(4 * sizeof(double), stream));  // [0]: potrf status (int), [2..3]: pivot range
  double* Z = (double*)zbuf.ptr;
  ZP_TRY(launch_walk(plan, r, theta, P, 0, Z, nullptr, stream));
  const double* Yuse = Y;
  if (w) {
    ZP_TRY(ybuf.alloc((size_t)P * S * sizeof(double), stream));
    scale_rows_kernel<<<1024, 256, 0, stream>>>(Z, J, P, w);
    scale_samples_kernel<<<1024, 256, 0, stream>>>(Y, (double*)ybuf.ptr, P, S, w);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "weight scaling launch");
    Yuse = (const double*)ybuf.ptr;
  }
  const double one = 1.0, zero = 0.0;
  if (emulated) {
    // Gram[i][j] = sum_p Z[i][p] Z[j][p] (exactly symmetric: both operands carry the same
    // scales and slices); RHS column-major J x S = row-major [S][J]: rhs[s][j] = sum_p Y[p][s] Z[j][p].
    ZP_TRY(emulated_gemm_fp64(J, J, P, Z, P, 1, Z, P, 1, (double*)gram.ptr, J, stream));
    ZP_TRY(emulated_gemm_fp64(S, J, P, Yuse, 1, S, Z, P, 1, (double*)rhs.ptr, J, stream));
  } else {
    // Z row-major [J][P] is column-major P x J (Zc).  Gram = Zc^T Zc: a full DGEMM (cuBLAS's
    // DSYRK measured three times slower for these shapes), of which potrf reads the lower half.
    if (cublasDgemm_64(blas, CUBLAS_OP_T, CUBLAS_OP_N, J, J, P, &one, Z, P, Z, P, &zero, (double*)gram.ptr, J) !=
        CUBLAS_STATUS_SUCCESS)
      return set_error(ZP_ERR_CUDA, "cublasDgemm (Gram) failed");
    // RHS (column-major J x S) = Zc^T (J x P) * Yc^T (P x S), Y row-major [P][S] = column-major S x P.
    if (cublasDgemm_64(blas, CUBLAS_OP_T, CUBLAS_OP_T, J, S, P, &one, Z, P, Yuse, S, &zero, (double*)rhs.ptr, J) !=
        CUBLAS_STATUS_SUCCESS)
      return set_error(ZP_ERR_CUDA, "cublasDgemm failed");
  }
  if (ridge > 0.0) {
    add_ridge_kernel<<<(unsigned)((J + 255) / 256), 256, 0, stream>>>((double*)gram.ptr, J, ridge);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "add_ridge_kernel launch");
  }
  int lwork = 0;
  if (cusolverDnDpotrf_bufferSize(sol, CUBLAS_FILL_MODE_LOWER, (int)J, (double*)gram.ptr, (int)J, &lwork) !=
      CUSOLVER_STATUS_SUCCESS)
    return set_error(ZP_ERR_CUDA, "cusolverDnDpotrf_bufferSize failed");
  ScratchBuffer work;
  ZP_TRY(work.alloc((size_t)std::max(lwork, 1) * sizeof(double), stream));
  if (cusolverDnDpotrf(sol, CUBLAS_FILL_MODE_LOWER, (int)J, (double*)gram.ptr, (int)J, (double*)work.ptr, lwork,
                       (int*)info.ptr) != CUSOLVER_STATUS_SUCCESS)
    return set_error(ZP_ERR_CUDA, "cusolverDnDpotrf failed");
  pivot_range_kernel<<<1, 256, 0, stream>>>((const double*)gram.ptr, J, (double*)info.ptr + 2);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "pivot_range_kernel launch");
  if (cusolverDnDpotrs(sol, CUBLAS_FILL_MODE_LOWER, (int)J, (int)S, (double*)gram.ptr, (int)J, (double*)rhs.ptr,
                       (int)J, (int*)info.ptr) != CUSOLVER_STATUS_SUCCESS)
    return set_error(ZP_ERR_CUDA, "cusolverDnDpotrs failed");
  // coeffs row-major [J][S] = column-major S x J = transpose of the J x S solution.
  if (cublasDgeam(blas, CUBLAS_OP_T, CUBLAS_OP_N, (int)S, (int)J, &one, (double*)rhs.ptr, (int)J, &zero, coeffs,
                  (int)S, coeffs, (int)S) != CUBLAS_STATUS_SUCCESS)
    return set_error(ZP_ERR_CUDA, "cublasDgeam failed");
  double h_info[4] = {0, 0, 0, 0};
  if ((e = cudaMemcpyAsync(h_info, info.ptr, sizeof(h_info), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return cuda_error(e, "reading the factorisation status");
  int status = 0;
  memcpy(&status, h_info, sizeof(int));
  // A rank-deficient normal matrix can factor with tiny positive pivots in floating point;
  // a squared-pivot ratio below 1e-14 (condition number above ~1e14) is reported as singular.
  if (status != 0 || !(h_info[2] > 1e-14 * h_info[3]))
    return set_error(ZP_ERR_INVALID_ARG, "normal matrix not positive definite (potrf status " + std::to_string(status) +
                                             ", squared pivot ratio " + std::to_string(h_info[2] / h_info[3]) +
                                             "): fewer independent points than modes, or duplicated modes; add a "
                                             "ridge");
  return ZP_OK;
}

}  // namespace zp

using namespace zp;

extern "C" {

zp_status zp_series_fit_plan(const zp_plan* plan, const double* r, const double* theta, const double* weights,
                             int64_t n_points, const double* samples, int64_t n_sets, double ridge, double* coeffs,
                             void* stream) {
  return zp_series_fit_plan_prec(plan, r, theta, weights, n_points, samples, n_sets, ridge, coeffs, ZP_PREC_FP64,
                                 stream);
}

zp_status zp_series_fit_plan_prec(const zp_plan* plan, const double* r, const double* theta, const double* weights,
                                  int64_t n_points, const double* samples, int64_t n_sets, double ridge,
                                  double* coeffs, zp_precision prec, void* stream) {
  clear_error();
  if (prec != ZP_PREC_FP64 && prec != ZP_PREC_FP64_EMULATED)
    return set_error(ZP_ERR_INVALID_ARG, "the fit takes ZP_PREC_FP64 or ZP_PREC_FP64_EMULATED");
  ZP_TRY(check_plan_device(plan));
  if (n_points < 0 || n_sets < 0) return set_error(ZP_ERR_INVALID_ARG, "negative size");
  if (!(ridge >= 0.0)) return set_error(ZP_ERR_INVALID_ARG, "ridge must be >= 0");
  if (plan->n_modes > 46340) return set_error(ZP_ERR_UNSUPPORTED, "fit supports at most 46340 modes");
  if (plan->n_modes == 0 || n_sets == 0) return ZP_OK;
  if (n_points == 0) return set_error(ZP_ERR_INVALID_ARG, "no points to fit");
  ZP_TRY(check_device_array(r, "r", 8));
  ZP_TRY(check_device_array(theta, "theta", 8));
  ZP_TRY(check_device_array(samples, "samples", 8));
  ZP_TRY(check_device_array(coeffs, "coeffs", 8));
  if (weights) ZP_TRY(check_device_array(weights, "weights", 8));
  if (n_sets > 0x7fffffff || plan->n_modes * n_sets > 0x7fffffffLL)
    return set_error(ZP_ERR_UNSUPPORTED, "fit output too large");
  return series_fit_fp64(plan, r, theta, weights, n_points, samples, n_sets, ridge, coeffs, (cudaStream_t)stream,
                         prec == ZP_PREC_FP64_EMULATED);
}

zp_status zp_series_fit(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r, const double* theta,
                        const double* weights, int64_t n_points, const double* samples, int64_t n_sets, double ridge,
                        double* coeffs, void* stream) {
  clear_error();
  std::shared_ptr<const zp_plan> held;
  ZP_TRY(cached_plan(n, m, n_modes, &held));
  const zp_plan* plan = held.get();
  return zp_series_fit_plan(plan, r, theta, weights, n_points, samples, n_sets, ridge, coeffs, stream);
}

}  // extern "C"
