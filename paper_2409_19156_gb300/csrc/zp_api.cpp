// C ABI entry points for the radial / basis evaluation and shared argument checks.
#include <cstdint>
#include <string>

#include "zp_api_common.h"

namespace zp {

zp_status check_device_array(const void* ptr, const char* name, size_t align) {
  if (!ptr) return set_error(ZP_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if ((uintptr_t)ptr % align != 0) {
    return set_error(ZP_ERR_INVALID_ARG, std::string(name) + " is not " + std::to_string(align) + "-byte aligned");
  }
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(ZP_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
  }
  if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr.type == cudaMemoryTypeDevice && attr.device != dev) {
      return set_error(ZP_ERR_INVALID_ARG, std::string(name) + " lives on device " + std::to_string(attr.device) +
                                               ", not the current device " + std::to_string(dev));
    }
    return ZP_OK;
  }
  // Pinned host memory mapped at the same address (cudaHostAlloc / cudaHostRegister under
  // unified addressing): the kernels read or write it across the host link.
  if (attr.type == cudaMemoryTypeHost && attr.devicePointer == ptr) return ZP_OK;
  if (attr.type == cudaMemoryTypeHost && attr.devicePointer != nullptr)
    return set_error(ZP_ERR_INVALID_ARG, std::string(name) + " is pinned host memory mapped at another device address");
  return set_error(ZP_ERR_INVALID_ARG, std::string(name) + " is not device-accessible memory");
}

}  // namespace zp

using namespace zp;

static zp_status radial_common(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                               int32_t max_deriv, double* out, double* out_dtheta, void* stream, bool angular,
                               float* phase_ms = nullptr) {
  ZP_TRY(check_plan_device(plan));
  if (n_points < 0) return set_error(ZP_ERR_INVALID_ARG, "n_points < 0");
  if (max_deriv < 0 || max_deriv > 3) return set_error(ZP_ERR_DERIV_ORDER, "max_deriv must be 0..3");
  if (n_points == 0 || plan->n_modes == 0) return ZP_OK;
  ZP_TRY(check_device_array(r, "r", 8));
  if (angular) ZP_TRY(check_device_array(theta, "theta", 8));
  ZP_TRY(check_device_array(out, "out", 8));
  if (out_dtheta) ZP_TRY(check_device_array(out_dtheta, "out_dtheta", 8));
  return launch_walk(plan, r, angular ? theta : nullptr, n_points, max_deriv, out, angular ? out_dtheta : nullptr,
                     (cudaStream_t)stream, phase_ms);
}

extern "C" {

static zp_status zp_radial_plan_impl(const zp_plan* plan, const double* r, int64_t n_points, int32_t max_deriv, double* out,
                         void* stream) {
  clear_error();
  return radial_common(plan, r, nullptr, n_points, max_deriv, out, nullptr, stream, false);
}

zp_status zp_radial_plan(const zp_plan* plan, const double* r, int64_t n_points, int32_t max_deriv, double* out,
                         void* stream) {
  zp::NvtxRange zp_range_("zp_radial_plan");
  return zp::entry_finish("zp_radial_plan", stream, zp_radial_plan_impl(plan, r, n_points, max_deriv, out, stream));
}

zp_status zp_radial_plan_timed(const zp_plan* plan, const double* r, int64_t n_points, int32_t max_deriv, double* out,
                               void* stream, float* phase_ms) {
  clear_error();
  if (!phase_ms) return set_error(ZP_ERR_INVALID_ARG, "phase_ms is NULL");
  return radial_common(plan, r, nullptr, n_points, max_deriv, out, nullptr, stream, false, phase_ms);
}

static zp_status zp_radial_impl(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r, int64_t n_points,
                    int32_t max_deriv, double* out, void* stream) {
  clear_error();
  if (max_deriv < 0 || max_deriv > 3) return set_error(ZP_ERR_DERIV_ORDER, "max_deriv must be 0..3");
  if (n_points < 0) return set_error(ZP_ERR_INVALID_ARG, "n_points < 0");
  std::shared_ptr<const zp_plan> held;
  ZP_TRY(cached_plan(n, m, n_modes, &held));
  const zp_plan* plan = held.get();
  return radial_common(plan, r, nullptr, n_points, max_deriv, out, nullptr, stream, false);
}

zp_status zp_radial(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r, int64_t n_points,
                    int32_t max_deriv, double* out, void* stream) {
  zp::NvtxRange zp_range_("zp_radial");
  return zp::entry_finish("zp_radial", stream, zp_radial_impl(n, m, n_modes, r, n_points, max_deriv, out, stream));
}

static zp_status zp_basis_plan_impl(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                        int32_t max_deriv, double* out, double* out_dtheta, void* stream) {
  clear_error();
  return radial_common(plan, r, theta, n_points, max_deriv, out, out_dtheta, stream, true);
}

zp_status zp_basis_plan(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                        int32_t max_deriv, double* out, double* out_dtheta, void* stream) {
  zp::NvtxRange zp_range_("zp_basis_plan");
  return zp::entry_finish("zp_basis_plan", stream, zp_basis_plan_impl(plan, r, theta, n_points, max_deriv, out, out_dtheta, stream));
}

static zp_status zp_basis_impl(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r, const double* theta,
                   int64_t n_points, int32_t max_deriv, double* out, double* out_dtheta, void* stream) {
  clear_error();
  if (max_deriv < 0 || max_deriv > 3) return set_error(ZP_ERR_DERIV_ORDER, "max_deriv must be 0..3");
  if (n_points < 0) return set_error(ZP_ERR_INVALID_ARG, "n_points < 0");
  std::shared_ptr<const zp_plan> held;
  ZP_TRY(cached_plan(n, m, n_modes, &held));
  const zp_plan* plan = held.get();
  return radial_common(plan, r, theta, n_points, max_deriv, out, out_dtheta, stream, true);
}

zp_status zp_basis(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r, const double* theta,
                   int64_t n_points, int32_t max_deriv, double* out, double* out_dtheta, void* stream) {
  zp::NvtxRange zp_range_("zp_basis");
  return zp::entry_finish("zp_basis", stream, zp_basis_impl(n, m, n_modes, r, theta, n_points, max_deriv, out, out_dtheta, stream));
}

static zp_status zp_radial_per_mode_impl(const zp_plan* plan, const double* r, int64_t n_points, double* out, void* stream) {
  clear_error();
  ZP_TRY(check_plan_device(plan));
  if (n_points < 0) return set_error(ZP_ERR_INVALID_ARG, "n_points < 0");
  if (n_points == 0 || plan->n_modes == 0) return ZP_OK;
  ZP_TRY(check_device_array(r, "r", 8));
  ZP_TRY(check_device_array(out, "out", 8));
  return launch_per_mode(plan, r, n_points, out, (cudaStream_t)stream);
}

zp_status zp_radial_per_mode(const zp_plan* plan, const double* r, int64_t n_points, double* out, void* stream) {
  zp::NvtxRange zp_range_("zp_radial_per_mode");
  return zp::entry_finish("zp_radial_per_mode", stream, zp_radial_per_mode_impl(plan, r, n_points, out, stream));
}

}  // extern "C"
