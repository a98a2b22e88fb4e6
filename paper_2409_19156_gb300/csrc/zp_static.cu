// Allocation-free variant of the split-precision series (zp_series_eval_static).
//
// Some callers cannot allocate device memory at call time: code running inside a host
// callback or a custom allocator's hook, runtimes that reserve all device memory up front
// and forbid further cudaMalloc, or processes where allocation would serialise against other
// work.  This entry point needs no device allocation at all: the plan tables, the split
// coefficient tiles and the split basis slab live in one file-scope device array of
// ZP_STATIC_SCRATCH_BYTES that exists on every GPU that loads the library, until exit.
//
// Host code must not use the array's name as a device address (in host code it names a
// host-side stand-in).  The device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and passed to the kernels.
//
// Under CUDA's default lazy module loading the array's device memory is committed when the
// library's module is first loaded on a device, which can be this entry point's first call
// there: a caller that must not allocate at all later should make one small call (or set
// CUDA_MODULE_LOADING=EAGER) while allocation is still allowed.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "zp_api_common.h"
#include "zp_series_internal.h"

// The one static scratch array (ZP_STATIC_SCRATCH_BYTES on every device that loads the library).
static __device__ __align__(256) unsigned char g_zp_static_scratch[ZP_STATIC_SCRATCH_BYTES];

namespace zp {
namespace {

std::mutex g_static_mu;
std::vector<void*> g_static_addr;  // per device: device address of g_zp_static_scratch

// Device address of the static scratch on the current device (looked up on first use).
zp_status static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if ((int)g_static_addr.size() <= dev) g_static_addr.resize(dev + 1, nullptr);
  if (!g_static_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_zp_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
    g_static_addr[dev] = ptr;
  }
  *out = g_static_addr[dev];
  return ZP_OK;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace
}  // namespace zp

using namespace zp;

static zp_status zp_series_eval_static_impl(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r,
                                           const double* theta, int64_t n_points, const double* coeffs,
                                           int64_t n_sets, zp_precision prec, float* out, void* stream) {
  clear_error();
  if (prec != ZP_PREC_BF16X3 && prec != ZP_PREC_TF32)
    return set_error(ZP_ERR_INVALID_ARG, "zp_series_eval_static supports ZP_PREC_BF16X3 and ZP_PREC_TF32 only");
  if (n_points < 0 || n_sets < 0) return set_error(ZP_ERR_INVALID_ARG, "negative size");
  // Size bounds before any product of sizes is formed: the array bounds the coefficient tiles
  // (at least 64 bytes per mode and set) and so n_modes * n_sets; the output memset and the
  // kernels' int64 index arithmetic bound n_points * n_sets.
  if (n_modes > (int64_t)(ZP_STATIC_SCRATCH_BYTES / 64) || n_sets > (int64_t)(ZP_STATIC_SCRATCH_BYTES / 64) ||
      (n_modes > 0 && n_sets > (int64_t)(ZP_STATIC_SCRATCH_BYTES / 64) / n_modes))
    return set_error(ZP_ERR_INVALID_ARG, "n_modes * n_sets exceeds what ZP_STATIC_SCRATCH_BYTES can hold; use "
                                         "zp_series_eval instead");
  if (n_sets > 0 && n_points > (int64_t)(INT64_MAX / 16) / n_sets)
    return set_error(ZP_ERR_INVALID_ARG, "n_points * n_sets too large");
  // The call copies its plan tables from host memory that is freed on return, which a captured
  // graph would read again at every replay: stream capture is refused.
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cs);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone)
      return set_error(ZP_ERR_INVALID_ARG, "zp_series_eval_static cannot be captured in a CUDA graph (its tables "
                                           "come from host memory freed on return); call it outside capture");
  }
  // Host half of a plan: validation, columns, tables (host memory only).
  zp_plan plan;
  ZP_TRY(build_plan_host(n, m, n_modes, &plan));
  if (n_points == 0 || n_sets == 0) return ZP_OK;
  ZP_TRY(check_device_array(r, "r", 8));
  ZP_TRY(check_device_array(theta, "theta", 8));
  ZP_TRY(check_device_array(coeffs, "coeffs", 8));
  ZP_TRY(check_device_array(out, "out", 16));
  cudaStream_t st = (cudaStream_t)stream;
  if (n_modes == 0) {
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n_points * n_sets * sizeof(float), st);
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "cudaMemsetAsync");
  }
  // Layout of the static array: plan tables | coefficient tiles | basis slab.
  size_t offsets[kPlanSections];
  const size_t table_bytes = round_up(plan_device_layout(&plan, offsets), 1024);
  size_t b_bytes = 0, tile_bytes = 0;
  const size_t need = table_bytes + round_up(split_scratch_bytes(prec, n_modes, n_sets, &b_bytes, &tile_bytes), 1024);
  if (need > (size_t)ZP_STATIC_SCRATCH_BYTES) {
    return set_error(ZP_ERR_INVALID_ARG,
                     "problem needs " + std::to_string(need) + " bytes of static scratch (tables, coefficient tiles "
                     "and one 128-point basis tile) but ZP_STATIC_SCRATCH_BYTES is " +
                         std::to_string((size_t)ZP_STATIC_SCRATCH_BYTES) + "; use zp_series_eval instead");
  }
  void* base = nullptr;
  ZP_TRY(static_scratch_address(&base));
  unsigned char* bytes = (unsigned char*)base;
  // Tables: pageable host -> device copies on the caller's stream (ordered after any
  // earlier call on that stream, which may still be reading the previous tables).
  ZP_TRY(plan_upload(&plan, bytes, st, true));
  SplitScratch sc;
  sc.b = bytes + table_bytes;
  sc.b_bytes = round_up(b_bytes, 1024);
  sc.a = sc.b + sc.b_bytes;
  sc.a_bytes = (size_t)ZP_STATIC_SCRATCH_BYTES - table_bytes - sc.b_bytes;
  // Every byte of the coefficient tiles and of each basis tile is written before it is read
  // within this call, so nothing left by an earlier call needs clearing.
  return series_eval_split(&plan, r, theta, n_points, coeffs, n_sets, prec, out, st, nullptr, &sc);
}

extern "C" zp_status zp_series_eval_static(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r,
                                           const double* theta, int64_t n_points, const double* coeffs,
                                           int64_t n_sets, zp_precision prec, float* out, void* stream) {
  zp::NvtxRange zp_range_("zp_series_eval_static");
  return zp::entry_finish("zp_series_eval_static", stream, zp_series_eval_static_impl(n, m, n_modes, r, theta, n_points, coeffs, n_sets, prec, out, stream));
}
