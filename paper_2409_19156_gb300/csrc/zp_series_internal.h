// Declarations shared by the series translation units.
#pragma once

#include <mutex>

#include "zp_internal.h"

namespace zp {

// Per-device memo of a host-side launch parameter that never changes for a device (occupancy
// queries, function attributes), computed on the device's first use: these queries cost far
// more host time than a launch, and the library's calls are often issued back to back.
template <typename T>
struct DeviceMemo {
  std::mutex mu;
  bool have[64] = {};
  T val[64] = {};
  template <typename F>
  zp_status get(T* out, F&& compute) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return compute(out);
    std::lock_guard<std::mutex> lock(mu);
    if (have[dev]) {
      *out = val[dev];
      return ZP_OK;
    }
    const zp_status st = compute(out);
    if (st != ZP_OK) return st;
    val[dev] = *out;
    have[dev] = true;
    return ZP_OK;
  }
};

// Stream-ordered scratch: cudaMallocAsync on `stream`, cudaFreeAsync on the same stream
// when the object goes out of scope (after the work that uses it has been enqueued).
struct ScratchBuffer {
  void* ptr = nullptr;
  cudaStream_t stream = nullptr;
  ScratchBuffer() = default;
  ScratchBuffer(const ScratchBuffer&) = delete;
  ScratchBuffer& operator=(const ScratchBuffer&) = delete;
  ~ScratchBuffer();
  zp_status alloc(size_t bytes, cudaStream_t s);
};

zp_status series_eval_fp64(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                           const double* coeffs, int64_t S, double* out, cudaStream_t stream);
// Optional per-point second-order outputs of the adjoint for L = <G, F>: the 2x2 Hessian
// blocks (rr, rt, tt: NULL or [P]) and, for a tangent (v_r, v_theta) ([P] each, both or
// neither), the Hessian-vector product (hv_r, hv_theta: NULL or [P]).
struct HessOut {
  double* rr = nullptr;
  double* rt = nullptr;
  double* tt = nullptr;
  const double* v_r = nullptr;
  const double* v_theta = nullptr;
  double* hv_r = nullptr;
  double* hv_theta = nullptr;
  bool any() const { return rr || rt || tt || hv_r || hv_theta; }
};
// emulated: the contractions on the float64-accurate tensor-core GEMM (else cuBLAS DGEMM).
zp_status series_adjoint_fp64(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                              const double* coeffs, int64_t S, const double* G, double* grad_coeffs,
                              double* grad_r, double* grad_theta, cudaStream_t stream, const HessOut& ho,
                              bool emulated);
// Split-precision tensor-core series (BF16x3 or TF32, float32 output).
// Float64-accurate series by error-free slicing on the tensor cores (float64 output).
zp_status series_eval_emulated_fp64(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                                    const double* coeffs, int64_t S, double* out, cudaStream_t stream);
// Float64-accurate GEMM on the tensor cores by the same slicing:
//   C[m * ldc + n] = sum_k A[m * a_sm + k * a_sk] * B[n * b_sn + k * b_sk],  m < M, n < N.
// Error bound: about K 2^-54 max_k |A(m, k)| max_k |B(n, k)| per element.  Scratch is
// allocated stream-ordered on `stream`.  a_rowmax: NULL, or per row m of A the high word of
// max_k |A(m, k)| shifted left by 32 (as the walk's rowmax output gives it), used for A's row
// scales instead of a pass over A.
zp_status emulated_gemm_fp64(int64_t M, int64_t N, int64_t K, const double* A, int64_t a_sm, int64_t a_sk,
                             const double* B, int64_t b_sn, int64_t b_sk, double* C, int64_t ldc,
                             cudaStream_t stream, const unsigned long long* a_rowmax = nullptr);

// Caller-provided scratch for the split path: `b` holds the split coefficient tiles,
// `a` the split basis of as many point tiles as fit (at least one).
struct SplitScratch {
  uint8_t* a = nullptr;
  size_t a_bytes = 0;
  uint8_t* b = nullptr;
  size_t b_bytes = 0;
};
// Bytes of coefficient tiles (*b_bytes) and of one point tile of split basis (*tile_bytes);
// returns their sum (the least scratch the split path can run in).
size_t split_scratch_bytes(zp_precision prec, int64_t n_modes, int64_t n_sets, size_t* b_bytes, size_t* tile_bytes);

// phase_ms: NULL, or [3] receiving the summed CUDA-event times of the coefficient split,
// the basis split and the GEMM launches (the call then synchronises the stream).
zp_status series_eval_split(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                            const double* coeffs, int64_t S, zp_precision prec, float* out,
                            cudaStream_t stream, float* phase_ms = nullptr,
                            const SplitScratch* preset = nullptr);

}  // namespace zp
