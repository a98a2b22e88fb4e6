// Argument-check helpers shared by the entry-point translation units.
#pragma once

#include "zp_internal.h"

#define ZP_TRY(expr)                    \
  do {                                  \
    zp_status zp_try_s_ = (expr);       \
    if (zp_try_s_ != ZP_OK) return zp_try_s_; \
  } while (0)

namespace zp {
// ZP_OK when ptr is non-NULL, `align`-byte aligned and reachable from the current device
// (device, managed or mapped pinned host memory); otherwise ZP_ERR_INVALID_ARG.
zp_status check_device_array(const void* ptr, const char* name, size_t align);
}  // namespace zp
