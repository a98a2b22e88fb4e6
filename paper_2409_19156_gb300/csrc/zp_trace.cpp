// Tracing and debug checks of the C ABI: NVTX ranges around every compute entry point and the
// ZP_DEBUG levels (see zp_api_common.h).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdio>
#include <cstdlib>
#include <string>

#include "zp_api_common.h"
#include "zp_fused.h"

namespace zp {

zp_status split_error_word(unsigned int* value, bool reset);

int debug_level() {
  static const int level = [] {
    const char* v = std::getenv("ZP_DEBUG");
    return v ? std::atoi(v) : 0;
  }();
  return level;
}

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

zp_status entry_finish(const char* name, void* stream, zp_status st) {
  const int level = debug_level();
  if (level <= 0) return st;
  if (st == ZP_OK) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      const std::string what = std::string(name) + " (ZP_DEBUG check)";
      cudaError_t e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) {
        st = cuda_error(e, what.c_str());
      } else {
        unsigned int a = 0, b = 0;
        if (split_error_word(&a, false) == ZP_OK && fused_error_word(&b, false) == ZP_OK && (a || b))
          st = set_error(ZP_ERR_TIMEOUT, what + ": a bounded device wait gave up");
      }
    } else {
      cudaGetLastError();
    }
  }
  if (level >= 2) std::fprintf(stderr, "[zp] %s -> %d%s%s\n", name, (int)st, st ? ": " : "", st ? zp_last_error() : "");
  return st;
}

}  // namespace zp
