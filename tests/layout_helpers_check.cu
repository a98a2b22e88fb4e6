// Host driver for tests/test_layout_helpers.py: prints the library's host-callable layout and
// conversion helpers for the inputs the test passes, so that the test can compare them with
// independent definitions.  No GPU is touched.
//   stdin: lines "t <hex64>" (trunc_float_bits of that float64 bit pattern) or "s <rowbytes>"
//          (every swizzled offset of a 256-row tile of 2- and 4-byte elements).
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "zp_internal.h"
#include "zp_ptx.cuh"

template <uint32_t ROW>
static void offsets() {
  for (uint32_t r = 0; r < 256; ++r)
    for (uint32_t k = 0; k < ROW / 2; ++k) std::printf("%u\n", zp::ptx::sw_offset_b16<ROW>(r, k));
  for (uint32_t r = 0; r < 256; ++r)
    for (uint32_t k = 0; k < ROW / 4; ++k) std::printf("%u\n", zp::ptx::sw_offset_b32<ROW>(r, k));
}

int main() {
  char op[8];
  while (std::scanf("%7s", op) == 1) {
    if (op[0] == 't') {
      uint64_t b = 0;
      if (std::scanf("%" SCNx64, &b) != 1) return 1;
      std::printf("%08x\n", zp::trunc_float_bits((uint32_t)(b >> 32), (uint32_t)b));
    } else if (op[0] == 's') {
      unsigned row = 0;
      if (std::scanf("%u", &row) != 1) return 1;
      if (row == 128) offsets<128>();
      else if (row == 64) offsets<64>();
      else return 1;
    }
  }
  return 0;
}
