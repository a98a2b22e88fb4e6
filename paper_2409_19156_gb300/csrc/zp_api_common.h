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

namespace zp {
// Debug-check level from the environment variable ZP_DEBUG (read once per process): 0 (the
// default) adds nothing; 1 synchronises the caller's stream after every compute entry point
// (outside stream capture) and turns an asynchronous CUDA error or a bounded device wait that
// gave up into that call's status; 2 also prints one line per call to stderr.
int debug_level();
// Ends a compute entry point: NVTX range closed by the caller's scope; with ZP_DEBUG >= 1 the
// checks above.  Returns the status to hand to the caller.
zp_status entry_finish(const char* name, void* stream, zp_status st);
// An NVTX range around one entry point (visible in Nsight Systems / Compute timelines).
struct NvtxRange {
  explicit NvtxRange(const char* name);
  ~NvtxRange();
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace zp
