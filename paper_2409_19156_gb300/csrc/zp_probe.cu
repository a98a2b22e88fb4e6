// Float64 issue-rate probe: the denominator of the float64 roofline of the recursion kernels.
//
// GB300's float64 rate is not in the vendor's usual tables, and the recursion kernels are
// bound by it, so the library measures it: every thread runs kChains independent dependent
// chains of one float64 operation (FMA, multiply or add) for `iters` rounds, with enough
// resident warps per SM to cover the pipe's latency.  The result is reported two ways:
//   - operations per second, from CUDA events around the launch, and
//   - lanes per SM per clock, from the SM cycle counter (clock64) read by every CTA at its
//     start and end, which does not depend on the clock the GPU ran at.
#include <cuda_runtime.h>

#include <vector>

#include "zp_api_common.h"

namespace zp {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 16;
constexpr int kUnroll = 4;  // rounds per loop trip (loop overhead off the float64 issue path)

// OP 0: x = fma(a, x, b); OP 1: x = x * a; OP 2: x = x + a, with a and b in registers shared by
// all chains (the recursion kernels' pattern: a step's coefficient feeds every Taylor lane).
// Three distinct 64-bit register operands per instruction (per-chain y, z) measured 1.68
// lanes/SM/clk, a and b from the constant bank 1.69: the register reads, not the float64 pipe,
// then limit the rate.  The values keep every chain finite and away from subnormals for any
// iteration count; the final values go to `sink` so the chains cannot be removed.
template <int OP>
__global__ void __launch_bounds__(kProbeThreads) fp64_probe_kernel(int iters, double a, double b, double* sink,
                                                                   long long* cycles) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  // Runtime values (not foldable into immediates or constant-bank operands).
  const double ar = a * (1.0 + 1e-15 * (threadIdx.x & 1)), br = b * (1.0 + 1e-15 * (threadIdx.x & 2));
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll kUnroll
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (OP == 0) {
        x[c] = fma(ar, x[c], br);
      } else if constexpr (OP == 1) {
        x[c] = x[c] * ar;
      } else {
        x[c] = x[c] + ar;
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) sink[threadIdx.x] = s;  // never true for these constants
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace zp

using namespace zp;

extern "C" ZP_API zp_status zp_probe_fp64(int32_t op, int32_t iters, void* stream, double* result) {
  clear_error();
  if (op < 0 || op > 2) return set_error(ZP_ERR_INVALID_ARG, "op must be 0 (FMA), 1 (multiply) or 2 (add)");
  if (iters < kUnroll || iters > (1 << 24) || iters % kUnroll != 0)
    return set_error(ZP_ERR_INVALID_ARG, "iters must be a multiple of 4 in 4..2^24");
  if (!result) return set_error(ZP_ERR_INVALID_ARG, "result is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_error(e, "device query");
  // Resident CTAs per SM of the chosen kernel: one full wave, every SM equally loaded.
  void (*kern)(int, double, double, double*, long long*) =
      op == 0 ? fp64_probe_kernel<0> : (op == 1 ? fp64_probe_kernel<1> : fp64_probe_kernel<2>);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kProbeThreads, 0);
  if (e != cudaSuccess) return cuda_error(e, "occupancy query");
  per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
  const int blocks = sms * per_sm;
  double* sink = nullptr;
  long long* cycles = nullptr;
  e = cudaMallocAsync(&sink, kProbeThreads * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&cycles, blocks * sizeof(long long), st);
  if (e != cudaSuccess) {
    if (sink) cudaFreeAsync(sink, st);
    return cuda_error(e, "probe scratch");
  }
  const double a = op == 0 ? 0.999999 : (op == 1 ? 0.9999999999 : 1e-9), b = 1e-6;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  kern<<<blocks, kProbeThreads, 0, st>>>(16, a, b, sink, cycles);  // warm-up
  cudaEventRecord(e0, st);
  kern<<<blocks, kProbeThreads, 0, st>>>(iters, a, b, sink, cycles);
  cudaEventRecord(e1, st);
  e = cudaGetLastError();
  std::vector<long long> cyc(blocks);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cyc.data(), cycles, blocks * sizeof(long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  cudaFreeAsync(cycles, st);
  if (e != cudaSuccess) return cuda_error(e, "fp64 probe");
  long long max_cyc = 1;
  for (long long c : cyc) max_cyc = c > max_cyc ? c : max_cyc;
  const double ops = (double)blocks * kProbeThreads * kChains * (double)iters;
  result[0] = ops;
  result[1] = ms;
  result[2] = ops / ((double)ms * 1e-3);                // operations per second
  result[3] = ops / ((double)sms * (double)max_cyc);    // lanes per SM per clock
  result[4] = (double)max_cyc / ((double)ms * 1e-3) * 1e-6;  // implied SM clock, MHz
  result[5] = (double)sms;
  return ZP_OK;
}
